"""Checksums of small seeded inputs (synth only: Philox streams, Gaussian fields,
the quenched heatbath).  They let any machine verify that it regenerates the
same bits, which the workloads rely on (their fields are regenerated, not
shipped).  usage: python tests/golden/make_synth_checksums.py"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import synth  # noqa: E402

CASES = {
    "gauge_4x4x4x4_b6_s10_or4_seed3": dict(L=(4, 4, 4, 4), beta=6.0, sweeps=10, n_or=4, seed=3),
    "gauge_4x2x4x6_b5.7_s6_or2_seed9": dict(L=(4, 2, 4, 6), beta=5.7, sweeps=6, n_or=2, seed=9),
}


def compute():
    out = {}
    for name, c in CASES.items():
        U = synth.gauge_field(c["L"], beta=c["beta"], sweeps=c["sweeps"], n_or=c["n_or"], seed=c["seed"], cache=False)
        out[name] = {"sha1": synth.checksum(U), "plaquette": synth.plaquette(U, c["L"])}
    out["gaussian_spinor_4x4x4x4_seed5_stream2"] = {"sha1": synth.checksum(synth.gaussian_spinor((4, 4, 4, 4), 5, 2))}
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_checksums.json")
    json.dump(compute(), open(path, "w"), indent=1)
    print(open(path).read())

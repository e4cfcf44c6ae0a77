"""Resource budget of the hot kernels, checked at build time (no GPU): ptxas's
report (-Xptxas -v) for the coarse CGNR kernels, which run one 512-thread CTA
per SM and so have at most 128 registers per thread, and for the fine operator.
A spill or a local-memory array in these kernels costs latency on every
stencil of every CG iteration; this test makes such a regression visible when
the library is compiled, before it is run."""
import os
import re
import shutil
import subprocess

import pytest

from paper_1005_3043_gb300 import build as wbuild


def ptxas_report(source):
    nvcc = wbuild._nvcc()
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = os.path.join(wbuild.BUILD, "resources_" + source.replace(".cu", ".o"))
    os.makedirs(wbuild.BUILD, exist_ok=True)
    cmd = [nvcc, *wbuild.ARCH, "-O3", "-std=c++17", "-Xptxas", "-v", "-I", os.path.join(wbuild.ROOT, "include"),
           "-I", wbuild.CSRC, "-c", os.path.join(wbuild.CSRC, source), "-o", out]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-2000:]
    report = {}
    name = None
    for line in res.stderr.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and name:
            report.setdefault(name, {}).update(stack=int(m.group(1)), spill_st=int(m.group(2)),
                                               spill_ld=int(m.group(3)))
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and name:
            report.setdefault(name, {})["regs"] = int(m.group(1))
    return report


@pytest.fixture(scope="module")
def cgls():
    return ptxas_report("kernels_cgls.cu")


# k_cgls_onchip<H16, TM>: TM 0 operator in shared memory, 1 tensor memory with
# CUDA-core products, 2 tensor memory with tensor-core products
CGLS = {"_ZN3wmg13k_cgls_onchipILb1ELi2EEEvNS_8CglsArgsE": "FP16, tensor-core products",
        "_ZN3wmg13k_cgls_onchipILb1ELi1EEEvNS_8CglsArgsE": "FP16, CUDA-core products",
        "_ZN3wmg13k_cgls_onchipILb0ELi1EEEvNS_8CglsArgsE": "FP32, CUDA-core products"}


@pytest.mark.parametrize("kernel", sorted(CGLS))
def test_coarse_cgnr_kernels_fit_one_cta_per_sm_without_spills(cgls, kernel):
    r = cgls[kernel]
    assert r["regs"] <= 128, (CGLS[kernel], r)            # 512 threads x 128 registers = the SM's file
    assert r["spill_st"] == 0 and r["spill_ld"] == 0, (CGLS[kernel], r)
    # the 32-byte frame holds the kernel's small fixed arrays; an accumulator
    # tile indexed at run time would add 128 bytes and more
    assert r["stack"] <= 32, (CGLS[kernel], r)


def test_fine_operator_spills_bounded():
    rep = ptxas_report("kernels_fine.cu")
    dslash = {k: v for k, v in rep.items() if "k_dslash" in k}
    assert dslash, "no k_dslash instantiation found in the ptxas report"
    for k, v in dslash.items():
        assert v["spill_st"] <= 128 and v["spill_ld"] <= 128, (k, v)

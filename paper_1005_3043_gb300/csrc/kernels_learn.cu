// The learned setup: a gauge-covariant parallel-transport convolution network
// that maps the links and random starts to prototypes for the adaptive setup
// (it stands in for the random-start relaxation that begins the Sec. IV setup,
// itself a polynomial in the hopping term of eq. 2).
//
// One layer:  out[a](x) = sum_b sum_d W[a][b][d] (T_d in[b])(x), d = 0 the site,
// 1 + 2 mu / 2 + 2 mu the neighbours x + mu / x - mu, (T_{+mu} p)(x) = U_mu(x)
// p(x + mu), (T_{-mu} p)(x) = U_mu(x - mu)^dag p(x - mu), the antiperiodic sign
// on hops across the t boundary; W[a][b][d] a 4x4 complex spin matrix.
// Activations: channel-major fine vectors in the internal layout
// T2 v[c][X][k 12][l]; weights W[a][b][d][s][t] complex FP32.
// The input gradient of a layer is the same layer with the weights
// W'[b][a][rev d] = W[a][b][d]^dag (T_{+mu}^dag = T_{-mu}), so one kernel
// serves both passes.
#include <algorithm>

#include "mg_launch.h"

namespace wmg {

constexpr int kNnThreads = 128;

// (T_d p)(x) for one channel: p read at the neighbour, colour-transported
template <int D>
__device__ __forceinline__ void nn_transport(cx<float> (&t)[4][3], const float2* __restrict__ in, const float2* __restrict__ U,
                                             const Geom& g, int X, int l, const int (&lc)[4], const int (&xc)[4]) {
    int Xn = X, ln = l;
    bool flip = false;
    if (D > 0) neighbour(g, X, l, lc, xc, (D - 1) >> 1, (D & 1) ? 1 : -1, Xn, ln, flip);
    cx<float> p[4][3];
    const float2* src = in + (size_t)Xn * 12 * g.Vb + ln;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) p[s][c] = ldg<float>(src + (3 * s + c) * g.Vb);
    if (D == 0) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) t[s][c] = p[s][c];
        return;
    }
    constexpr int MU = (D - 1) >> 1;
    constexpr bool FWD = (D & 1) != 0;
    const size_t ls = FWD ? ((size_t)MU * g.Vc + X) : ((size_t)MU * g.Vc + Xn);
    const float2* u = U + ls * 9 * g.Vb + (FWD ? l : ln);
    cx<float> m[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) m[e] = ldg<float>(u + (size_t)e * g.Vb);
    const float sg = flip ? -1.f : 1.f;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<float> acc(0, 0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (FWD) cmad(acc, m[3 * a + b], p[s][b]);
                else cmadc(acc, m[3 * b + a], p[s][b]);
            }
            t[s][a] = sg * acc;
        }
}

// Four threads per site, one per spin s (lanes 4i .. 4i+3 of a warp share a
// site).  For every input channel b and direction d, thread s transports its
// own spin row of in[b] (3 colours: 3 loads, one link, 9 complex multiply-adds),
// the four rows are exchanged by warp shuffles, and the thread adds
// W[a][b][d][s][t] (T_d in[b])[t] for every output channel a into its
// registers: each transport is formed once instead of once per output channel.
// The layer's weights sit in shared memory (W[a][b][d][s][t], cout * cin * 144
// complex).
constexpr int kNnMaxCout = 8;
__global__ void __launch_bounds__(kNnThreads) k_nn_layer(float2* __restrict__ out, const float2* __restrict__ in,
                                                         const float2* __restrict__ W, const float2* __restrict__ U,
                                                         Geom g, int cin, int cout) {
    extern __shared__ float2 sW[];
    for (int i = threadIdx.x; i < cout * cin * 144; i += blockDim.x) sW[i] = W[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, sp = lane & 3, gbase = lane & ~3;
    const long long site = blockIdx.x * (long long)(blockDim.x >> 2) + (threadIdx.x >> 2);
    const bool live = site < g.V;
    const long long s = live ? site : g.V - 1;   // idle lanes shadow the last site (for the shuffles)
    const int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
    int lc[4], xc[4];
    local_coords(g, l, lc);
    coarse_coords(g, X, xc);
    const size_t chan = (size_t)g.V * 12;
    cx<float> acc[kNnMaxCout][3];
#pragma unroll
    for (int a = 0; a < kNnMaxCout; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[a][c] = cx<float>(0, 0);
    for (int b = 0; b < cin; ++b) {
        const float2* inb = in + (size_t)b * chan;
#pragma unroll 1
        for (int d = 0; d < 9; ++d) {
            int Xn = X, ln = l;
            bool flip = false;
            if (d > 0) neighbour(g, X, l, lc, xc, (d - 1) >> 1, (d & 1) ? 1 : -1, Xn, ln, flip);
            cx<float> p[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) p[c] = ldg<float>(inb + ((size_t)Xn * 12 + 3 * sp + c) * g.Vb + ln);
            cx<float> t[3];
            if (d == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) t[c] = p[c];
            } else {
                const int mu = (d - 1) >> 1;
                const bool fwd = (d & 1) != 0;
                const size_t ls = fwd ? ((size_t)mu * g.Vc + X) : ((size_t)mu * g.Vc + Xn);
                const float2* u = U + ls * 9 * g.Vb + (fwd ? l : ln);
                cx<float> m[9];
#pragma unroll
                for (int e = 0; e < 9; ++e) m[e] = ldg<float>(u + (size_t)e * g.Vb);
                const float sg = flip ? -1.f : 1.f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cx<float> q(0, 0);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        if (fwd) cmad(q, m[3 * a + c], p[c]);
                        else cmadc(q, m[3 * c + a], p[c]);
                    }
                    t[a] = sg * q;
                }
            }
            // the four spin rows of the transported vector, from the site's four lanes
            cx<float> tt[4][3];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    tt[r][c].r = __shfl_sync(0xffffffffu, t[c].r, gbase + r);
                    tt[r][c].i = __shfl_sync(0xffffffffu, t[c].i, gbase + r);
                }
            const float2* wb = sW + ((size_t)b * 9 + d) * 16 + 4 * sp;   // W[a][b][d][sp][.] at + a * cin * 144
#pragma unroll
            for (int a = 0; a < kNnMaxCout; ++a) {
                if (a >= cout) break;
                const float2* w = wb + (size_t)a * cin * 144;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const cx<float> wv(w[r].x, w[r].y);
#pragma unroll
                    for (int c = 0; c < 3; ++c) cmad(acc[a][c], wv, tt[r][c]);
                }
            }
        }
    }
    if (!live) return;
#pragma unroll
    for (int a = 0; a < kNnMaxCout; ++a) {
        if (a >= cout) break;
        float2* o = out + (size_t)a * chan + ((size_t)X * 12 + 3 * sp) * g.Vb + l;
#pragma unroll
        for (int c = 0; c < 3; ++c) st<float>(o + (size_t)c * g.Vb, acc[a][c]);
    }
}

// ---------------------------------------------------------------- weight gradient
// part[blk][q][16], q = (a * cin + b) * 9 + d: sum over this CTA's sites and the
// colours of g[a](x)_s conj((T_d in[b])(x)_t), one thread per q
template <int D>
__device__ __forceinline__ void nn_wgrad_site(cx<float> (&acc)[16], const float2* __restrict__ gout,
                                              const float2* __restrict__ in, const float2* __restrict__ U,
                                              const Geom& g, int X, int l, const int (&lc)[4], const int (&xc)[4]) {
    cx<float> t[4][3];
    nn_transport<D>(t, in, U, g, X, l, lc, xc);
    const float2* gp = gout + (size_t)X * 12 * g.Vb + l;
    cx<float> gv[4][3];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) gv[s][c] = ldg<float>(gp + (3 * s + c) * g.Vb);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int tt = 0; tt < 4; ++tt)
#pragma unroll
            for (int c = 0; c < 3; ++c) cmadc(acc[4 * s + tt], t[tt][c], gv[s][c]);   // conj(t) g
}

constexpr int kNnWgradThreads = 288;   // parameter blocks per CTA (130 registers each)
__global__ void __launch_bounds__(kNnWgradThreads) k_nn_wgrad(float2* __restrict__ part, const float2* __restrict__ gout,
                                                              const float2* __restrict__ in,
                                                              const float2* __restrict__ U, Geom g, int cin, int cout) {
    const int q = blockIdx.y * blockDim.x + threadIdx.x, nq = cout * cin * 9;
    if (q >= nq) return;
    const int d = q % 9, b = (q / 9) % cin, a = q / (9 * cin);
    const size_t chan = (size_t)g.V * 12;
    const long long s0 = (long long)blockIdx.x * g.V / gridDim.x, s1 = (long long)(blockIdx.x + 1) * g.V / gridDim.x;
    cx<float> acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = cx<float>(0, 0);
    for (long long s = s0; s < s1; ++s) {
        const int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
        int lc[4], xc[4];
        local_coords(g, l, lc);
        coarse_coords(g, X, xc);
        const float2* go = gout + (size_t)a * chan;
        const float2* ib = in + (size_t)b * chan;
        switch (d) {
            case 0: nn_wgrad_site<0>(acc, go, ib, U, g, X, l, lc, xc); break;
            case 1: nn_wgrad_site<1>(acc, go, ib, U, g, X, l, lc, xc); break;
            case 2: nn_wgrad_site<2>(acc, go, ib, U, g, X, l, lc, xc); break;
            case 3: nn_wgrad_site<3>(acc, go, ib, U, g, X, l, lc, xc); break;
            case 4: nn_wgrad_site<4>(acc, go, ib, U, g, X, l, lc, xc); break;
            case 5: nn_wgrad_site<5>(acc, go, ib, U, g, X, l, lc, xc); break;
            case 6: nn_wgrad_site<6>(acc, go, ib, U, g, X, l, lc, xc); break;
            case 7: nn_wgrad_site<7>(acc, go, ib, U, g, X, l, lc, xc); break;
            default: nn_wgrad_site<8>(acc, go, ib, U, g, X, l, lc, xc); break;
        }
    }
    float2* o = part + ((size_t)blockIdx.x * nq + q) * 16;
#pragma unroll
    for (int k = 0; k < 16; ++k) o[k] = make_float2(acc[k].r, acc[k].i);
}
// G[q][k] += scale * sum over blocks of part[blk][q][k] (fixed order, FP64 sums)
__global__ void k_nn_wgrad_sum(double2* __restrict__ G, const float2* __restrict__ part, int nblk, int n, double scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double re = 0, im = 0;
    for (int b = 0; b < nblk; ++b) {
        const float2 v = part[(size_t)b * n + i];
        re += v.x;
        im += v.y;
    }
    G[i].x += scale * re;
    G[i].y += scale * im;
}

// ---------------------------------------------------------------- loss seed and optimiser
// g = r / vv - rr v / vv^2 with vv = scal[vslot], rr = scal[rslot]: the derivative of
// |r|^2 / |v|^2 with respect to conj(v) for r = (1 - P P^dag) v
__global__ void k_nn_seed(float2* __restrict__ gout, const float2* __restrict__ r, const float2* __restrict__ v, size_t n,
                          const double* __restrict__ scal, int vslot, int rslot) {
    const double vv = scal[vslot], rr = scal[rslot];
    const float a = (float)(1.0 / vv), b = (float)(rr / (vv * vv));
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 rv = r[i], vv2 = v[i];
        gout[i] = make_float2(a * rv.x - b * vv2.x, a * rv.y - b * vv2.y);
    }
}
// Adam on complex weights (real and imaginary parts as independent reals)
__global__ void k_nn_adam(float2* __restrict__ W, double2* __restrict__ Wm, const double2* __restrict__ G,
                          double2* __restrict__ m, double2* __restrict__ v, int n, double lr, double b1, double b2,
                          double eps, int t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    double2 gg = G[i], mm = m[i], vv = v[i], w = Wm[i];
    mm.x = b1 * mm.x + (1 - b1) * gg.x;
    mm.y = b1 * mm.y + (1 - b1) * gg.y;
    vv.x = b2 * vv.x + (1 - b2) * gg.x * gg.x;
    vv.y = b2 * vv.y + (1 - b2) * gg.y * gg.y;
    w.x -= lr * (mm.x / c1) / (sqrt(vv.x / c2) + eps);
    w.y -= lr * (mm.y / c1) / (sqrt(vv.y / c2) + eps);
    m[i] = mm;
    v[i] = vv;
    Wm[i] = w;
    if (W) W[i] = make_float2((float)w.x, (float)w.y);
}
// W'[b][a][rev d] = W[a][b][d]^dag: the weights of a layer's input-gradient pass
__global__ void k_nn_adjoint_weights(float2* __restrict__ Wt, const float2* __restrict__ W, int cin, int cout) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, n = cout * cin * 9 * 16;
    if (i >= n) return;
    const int k = i % 16, d = (i / 16) % 9, b = (i / 144) % cin, a = i / (144 * cin);
    const int s = k / 4, t = k % 4;
    const int rd = d == 0 ? 0 : ((d & 1) ? d + 1 : d - 1);
    const float2 w = W[i];
    Wt[(((size_t)b * cout + a) * 9 + rd) * 16 + 4 * t + s] = make_float2(w.x, -w.y);
}

// ---------------------------------------------------------------- launchers
cudaError_t nn_layer(float2* out, const float2* in, const float2* W, const float2* U, const Geom& g, int cin, int cout,
                     cudaStream_t st) {
    if (cout > kNnMaxCout) return cudaErrorInvalidValue;
    const size_t sm = sizeof(float2) * (size_t)cout * cin * 144;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_nn_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    const int sites_per_cta = kNnThreads / 4;
    note_launch();
    k_nn_layer<<<(unsigned)((g.V + sites_per_cta - 1) / sites_per_cta), kNnThreads, sm, st>>>(out, in, W, U, g, cin, cout);
    return cudaGetLastError();
}
int nn_wgrad_blocks(const Geom& g) {
    long long b = (g.V + 255) / 256;
    return (int)(b < 608 ? b : 608);
}
cudaError_t nn_wgrad(double2* G, float2* part, const float2* gout, const float2* in, const float2* U, const Geom& g,
                     int cin, int cout, double scale, cudaStream_t st) {
    const int nq = cout * cin * 9, nblk = nn_wgrad_blocks(g);
    const int thr = std::min(kNnWgradThreads, ((nq + 31) / 32) * 32);
    note_launch();
    k_nn_wgrad<<<dim3(nblk, (nq + thr - 1) / thr), thr, 0, st>>>(part, gout, in, U, g, cin, cout);
    note_launch();
    k_nn_wgrad_sum<<<(nq * 16 + 255) / 256, 256, 0, st>>>(G, part, nblk, nq * 16, scale);
    return cudaGetLastError();
}
void nn_seed(float2* gout, const float2* r, const float2* v, size_t n, const double* scal, int vslot, int rslot,
             cudaStream_t st) {
    note_launch();
    k_nn_seed<<<(int)std::min<size_t>((n + 255) / 256, (size_t)device_sm_count() * 16), 256, 0, st>>>(gout, r, v, n, scal, vslot, rslot);
}
void nn_adam(float2* W, double2* Wm, const double2* G, double2* m, double2* v, int n, double lr, double b1, double b2,
             double eps, int t, cudaStream_t st) {
    note_launch();
    k_nn_adam<<<(n + 255) / 256, 256, 0, st>>>(W, Wm, G, m, v, n, lr, b1, b2, eps, t);
}
void nn_adjoint_weights(float2* Wt, const float2* W, int cin, int cout, cudaStream_t st) {
    const int n = cout * cin * 144;
    note_launch();
    k_nn_adjoint_weights<<<(n + 255) / 256, 256, 0, st>>>(Wt, W, cin, cout);
}

}  // namespace wmg

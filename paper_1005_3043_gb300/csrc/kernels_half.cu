// FP16 storage of the fine level (MG_FP16 mode): the Wilson operator (eq. 2)
// and the MR smoother (Sec. III) on spinors stored as FP16 with one FP32 scale
// per site and links stored as FP16 (|U_ij| <= 1 for SU(3), no scale).
// Arithmetic is FP32 throughout; only storage is FP16.
//
// Half spinor layout: h[X][j 6][l] (uint2 = two __half2: components 2j and
// 2j+1 of the site, value / scale) and s[X][l] (the site's max |re|, |im|
// over its 24 reals; 0 for a zero site).  Links: U16[mu][X][j 5][l] (uint2:
// entries 2j and 2j+1 of the 3x3 matrix, the last half-word zero).  Pairs
// halve the load instructions per hop (6 + 5 instead of 12 + 9): the
// dslash is limited by dependent load rounds, not bytes.
#include <cuda_fp16.h>

#include "mg_launch.h"
#include "mg_wilson.cuh"

namespace wmg {

namespace {
constexpr int kHalfThreads = 128;
inline int half_grid(long long n) { return (int)((n + kHalfThreads - 1) / kHalfThreads); }

__device__ __forceinline__ cx<float> h2c(uint32_t w, float s) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w));
    return cx<float>(f.x * s, f.y * s);
}
__device__ __forceinline__ uint32_t c2h(float re, float im) {
    const __half2 q = __floats2half2_rn(re, im);
    return *reinterpret_cast<const uint32_t*>(&q);
}
// the factor 1 / |v| of a normalised basis vector, stored as a float in a
// double scalar (nullptr: 1); its site scales times this factor are the
// scales of the normalised vector
__device__ __forceinline__ float inv_norm(const double* f) { return f ? (float)*f : 1.f; }
// the 12 components of a site (6 pair words at stride Vb), times s
__device__ __forceinline__ void ld_site_h(const uint2* p, float s, int Vb, cx<float> (&v)[12]) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const uint2 w = __ldg(p + (size_t)j * Vb);
        v[2 * j] = h2c(w.x, s);
        v[2 * j + 1] = h2c(w.y, s);
    }
}
// write the 12 components of a site as FP16 pairs with a per-site scale;
// each stored (rounded) value is passed to use(k, value)
template <typename Use>
__device__ __forceinline__ void store_site_h(uint2* h, float* s, const cx<float> (&v)[12], int Vb, Use use) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].r), fabsf(v[k].i)));
    const float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        uint2 w;
        w.x = c2h(v[2 * j].r * inv, v[2 * j].i * inv);
        w.y = c2h(v[2 * j + 1].r * inv, v[2 * j + 1].i * inv);
        h[(size_t)j * Vb] = w;
        use(2 * j, h2c(w.x, m));
        use(2 * j + 1, h2c(w.y, m));
    }
    *s = m;
}
__device__ __forceinline__ void store_site_h(uint2* h, float* s, const cx<float> (&v)[12], int Vb) {
    store_site_h(h, s, v, Vb, [](int, cx<float>) {});
}

// one hop on FP16 storage (input spinor IN16: FP16 pairs + scale, else FP32)
template <int MU, bool FWD, bool IN16>
__device__ __forceinline__ void hop_h(cx<float> (&acc)[4][3], const void* __restrict__ in, const float* __restrict__ sin,
                                      float fin, const uint2* __restrict__ U, const Geom& g, int X, int l,
                                      const int (&lc)[4], const int (&xc)[4]) {
    int Xn, ln;
    bool flip;
    neighbour(g, X, l, lc, xc, MU, FWD ? 1 : -1, Xn, ln, flip);
    cx<float> p[4][3];
    cx<float>(&pf)[12] = reinterpret_cast<cx<float>(&)[12]>(p);
    if (IN16) {
        ld_site_h(reinterpret_cast<const uint2*>(in) + (size_t)Xn * 6 * g.Vb + ln,
                  __ldg(sin + (size_t)Xn * g.Vb + ln) * fin, g.Vb, pf);
    } else {
        const float2* b = reinterpret_cast<const float2*>(in) + (size_t)Xn * 12 * g.Vb + ln;
#pragma unroll
        for (int k = 0; k < 12; ++k) pf[k] = ldg<float>(b + (size_t)k * g.Vb);
    }
    cx<float> h[2][3];
    project<float, MU, FWD>(p, h);
    const uint2* u = FWD ? U + ((size_t)MU * g.Vc + X) * 5 * g.Vb + l : U + ((size_t)MU * g.Vc + Xn) * 5 * g.Vb + ln;
    cx<float> m[9];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const uint2 w = __ldg(u + (size_t)j * g.Vb);
        m[2 * j] = h2c(w.x, 1.f);
        if (2 * j + 1 < 9) m[2 * j + 1] = h2c(w.y, 1.f);
    }
    cx<float> w[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w[0][a] = cx<float>(0.f, 0.f);
        w[1][a] = cx<float>(0.f, 0.f);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (FWD) {
                cmad(w[0][a], m[3 * a + b], h[0][b]);
                cmad(w[1][a], m[3 * a + b], h[1][b]);
            } else {
                cmadc(w[0][a], m[3 * b + a], h[0][b]);
                cmadc(w[1][a], m[3 * b + a], h[1][b]);
            }
        }
    accumulate<float, MU, FWD>(acc, w, flip ? 0.5f : -0.5f);
}
}  // namespace

// out (FP16 + scale) = D in, or src - D in (HMODE_XMY), or D in with the MR
// dot products <q, in>, |q|^2 of the stored q (HMODE_MRDOT -> omega <q,r>/<q,q>)
enum { HMODE_PLAIN = 0, HMODE_XMY = 1, HMODE_MRDOT = 2 };

template <int MODE, bool IN16>
__global__ void __launch_bounds__(kHalfThreads, MODE == HMODE_MRDOT ? 6 : 7)
    k_dslash_h(uint2* __restrict__ out, float* __restrict__ sout, const void* __restrict__ in,
               const float* __restrict__ sin, const double* __restrict__ fnorm, const uint2* __restrict__ U,
               const float2* __restrict__ src, Geom g, float diag, double omega, Reduce R) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const float fin = IN16 ? inv_norm(fnorm) : 1.f;   // the input's site scales times fin
    float red[3] = {0.f, 0.f, 0.f};
    if (s < g.V) {
        const int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
        int lc[4], xc[4];
        local_coords(g, l, lc);
        coarse_coords(g, X, xc);
        const size_t self = (size_t)X * 12 * g.Vb + l;     // FP32 vectors
        const size_t self6 = (size_t)X * 6 * g.Vb + l;     // FP16 pair vectors
        const float sself = IN16 ? __ldg(sin + (size_t)X * g.Vb + l) * fin : 1.f;
        // the input at this site (re-read, cached, where the MR dots need it)
        auto self_in = [&](int k) -> cx<float> {
            if (IN16) {
                const uint2 w = __ldg(reinterpret_cast<const uint2*>(in) + self6 + (size_t)(k >> 1) * g.Vb);
                return h2c((k & 1) ? w.y : w.x, sself);
            }
            return ldg<float>(reinterpret_cast<const float2*>(in) + self + (size_t)k * g.Vb);
        };
        cx<float> acc[4][3];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[sp][c] = diag * self_in(3 * sp + c);
        hop_h<0, true, IN16>(acc, in, sin, fin, U, g, X, l, lc, xc);
        hop_h<0, false, IN16>(acc, in, sin, fin, U, g, X, l, lc, xc);
        hop_h<1, true, IN16>(acc, in, sin, fin, U, g, X, l, lc, xc);
        hop_h<1, false, IN16>(acc, in, sin, fin, U, g, X, l, lc, xc);
        hop_h<2, true, IN16>(acc, in, sin, fin, U, g, X, l, lc, xc);
        hop_h<2, false, IN16>(acc, in, sin, fin, U, g, X, l, lc, xc);
        hop_h<3, true, IN16>(acc, in, sin, fin, U, g, X, l, lc, xc);
        hop_h<3, false, IN16>(acc, in, sin, fin, U, g, X, l, lc, xc);
        cx<float>(&v)[12] = reinterpret_cast<cx<float>(&)[12]>(acc);   // component k = 3 spin + colour
        if (MODE == HMODE_XMY)
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] = ldg<float>(src + self + (size_t)k * g.Vb) - v[k];
        store_site_h(out + self6, sout + (size_t)X * g.Vb + l, v, g.Vb, [&](int k, cx<float> q) {
            if (MODE == HMODE_MRDOT) {
                const cx<float> r = self_in(k);
                red[0] += q.r * r.r + q.i * r.i;
                red[1] += q.r * r.i - q.i * r.r;
                red[2] += norm2(q);
            }
        });
    }
    if (MODE == HMODE_MRDOT) {
        float v3[3] = {red[0], red[1], red[2]};
        grid_reduce<3, float>(v3, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[3]) {
            const double f = t[2] > 0 ? omega / t[2] : 0.0;
            R.scal[S_MR_ALPHA] = f * t[0];
            R.scal[S_MR_ALPHA + 1] = f * t[1];
        });
    }
}

// e += alpha r;  r -= alpha q (update_r), r and q in FP16 storage, e FP32
__global__ void __launch_bounds__(kHalfThreads) k_mr_update_h(float2* __restrict__ e, uint2* __restrict__ r,
                                                               float* __restrict__ sr, const uint2* __restrict__ q,
                                                               const float* __restrict__ sq, Geom g, bool update_r,
                                                               const double* __restrict__ scal) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
    const size_t self = (size_t)X * 12 * g.Vb + l, self6 = (size_t)X * 6 * g.Vb + l;
    const cx<float> a((float)scal[S_MR_ALPHA], (float)scal[S_MR_ALPHA + 1]);
    cx<float> rv[12];
    ld_site_h(r + self6, sr[(size_t)X * g.Vb + l], g.Vb, rv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        cx<float> ei = ld<float>(e + self + (size_t)k * g.Vb);
        cmad(ei, a, rv[k]);
        st<float>(e + self + (size_t)k * g.Vb, ei);
    }
    if (update_r) {
        cx<float> qv[12];
        ld_site_h(q + self6, __ldg(sq + (size_t)X * g.Vb + l), g.Vb, qv);
#pragma unroll
        for (int k = 0; k < 12; ++k) rv[k] = rv[k] - a * qv[k];
        store_site_h(r + self6, sr + (size_t)X * g.Vb + l, rv, g.Vb);
    }
}

__global__ void k_to_half(uint2* __restrict__ h, float* __restrict__ sc, const float2* __restrict__ x, Geom g) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
    const size_t self = (size_t)X * 12 * g.Vb + l;
    cx<float> v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = ld<float>(x + self + (size_t)k * g.Vb);
    store_site_h(h + (size_t)X * 6 * g.Vb + l, sc + (size_t)X * g.Vb + l, v, g.Vb);
}
__global__ void k_from_half(float2* __restrict__ x, const uint2* __restrict__ h, const float* __restrict__ sc, Geom g) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
    const size_t self = (size_t)X * 12 * g.Vb + l;
    cx<float> v[12];
    ld_site_h(h + (size_t)X * 6 * g.Vb + l, sc[(size_t)X * g.Vb + l], g.Vb, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) st<float>(x + self + (size_t)k * g.Vb, v[k]);
}
// U16[mu][X][j][l] = (U[mu][X][2j][l], U[mu][X][2j+1][l]) rounded (entry 9 = 0)
__global__ void k_links_to_half(uint2* __restrict__ U16, const float2* __restrict__ U, Geom g) {
    const long long n = 4LL * g.Vc * 5 * g.Vb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long l = i % g.Vb, t = i / g.Vb;
        const int j = (int)(t % 5);
        const long long mx = t / 5;   // mu * Vc + X
        const float2* src = U + (mx * 9 + 2 * j) * g.Vb + l;
        uint2 w;
        w.x = c2h(src[0].x, src[0].y);
        w.y = (2 * j + 1 < 9) ? c2h(src[g.Vb].x, src[g.Vb].y) : 0u;
        U16[i] = w;
    }
}

// ---------------------------------------------------------------- GMRES basis in FP16 storage
// Vector j of the basis: pairs B[j][X][6][l] and per-site scales S[j][X][l] (the
// HalfSpinor layout); column j of the Hessenberg matrix in the scalars as in the
// FP32 smoother (rslot).  Normalising a vector only rescales its site scales.
namespace {
__device__ __forceinline__ int rslot_h(int j, int k) { return S_GCR_R + 2 * (k * K_MAX + j); }
}
template <int NJ>
__global__ void __launch_bounds__(kHalfThreads) k_h_multidot(const uint2* __restrict__ B, const float* __restrict__ S,
                                                              Geom g, int k, Reduce R) {
    __shared__ float fac[K_MAX];   // basis j < k is normalised through its stored norm
    for (int j = threadIdx.x; j < k && j < K_MAX; j += blockDim.x) fac[j] = inv_norm(R.scal + S_GMRES_F + j);
    __syncthreads();
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float a[2 * NJ];
#pragma unroll
    for (int j = 0; j < 2 * NJ; ++j) a[j] = 0.f;
    if (s < g.V) {
        const int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
        const size_t self6 = (size_t)X * 6 * g.Vb + l, V6 = (size_t)6 * g.V;
        cx<float> w[12];
        ld_site_h(B + (size_t)k * V6 + self6, S[(size_t)k * g.V + s], g.Vb, w);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            if (j < k) {
                cx<float> v[12];
                ld_site_h(B + (size_t)j * V6 + self6, S[(size_t)j * g.V + s] * fac[j], g.Vb, v);
                cx<float> t(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 12; ++q) cmadc(t, v[q], w[q]);
                a[2 * j] = t.r;
                a[2 * j + 1] = t.i;
            }
        }
    }
    grid_reduce<2 * NJ, float>(a, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[2 * NJ]) {
        for (int j = 0; j < k && j < NJ; ++j) {
            R.scal[rslot_h(j, k)] = t[2 * j];
            R.scal[rslot_h(j, k) + 1] = t[2 * j + 1];
        }
    });
}
// basis[k] -= sum_{j<k} h_jk basis[j] (h from the scalars), stored again in FP16
// with new site scales; h_{k,k-1} = |basis[k]| of the stored vector is recorded
// and normalises it: its readers scale its site scales by the float 1 / |basis[k]|
// (S_GMRES_F + k), the same float product a rescaling pass would have stored
__global__ void __launch_bounds__(kHalfThreads) k_h_orth(uint2* __restrict__ B, float* __restrict__ S, Geom g, int k,
                                                          Reduce R) {
    __shared__ double beta[2 * K_MAX];
    __shared__ float fac[K_MAX];
    for (int j = threadIdx.x; j < 2 * k; j += blockDim.x) beta[j] = R.scal[S_GCR_R + 2 * k * K_MAX + j];
    for (int j = threadIdx.x; j < k && j < K_MAX; j += blockDim.x) fac[j] = inv_norm(R.scal + S_GMRES_F + j);
    __syncthreads();
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float a = 0.f;
    if (s < g.V) {
        const int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
        const size_t self6 = (size_t)X * 6 * g.Vb + l, V6 = (size_t)6 * g.V;
        cx<float> w[12];
        ld_site_h(B + (size_t)k * V6 + self6, S[(size_t)k * g.V + s], g.Vb, w);
        for (int j = 0; j < k; ++j) {
            cx<float> v[12];
            ld_site_h(B + (size_t)j * V6 + self6, S[(size_t)j * g.V + s] * fac[j], g.Vb, v);
            const cx<float> b((float)beta[2 * j], (float)beta[2 * j + 1]);
#pragma unroll
            for (int q = 0; q < 12; ++q) w[q] = w[q] - b * v[q];
        }
        store_site_h(B + (size_t)k * V6 + self6, S + (size_t)k * g.V + s, w, g.Vb,
                     [&](int, cx<float> q) { a += norm2(q); });
    }
    float acc[1] = {a};
    grid_reduce<1, float>(acc, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) {
        const double nk = sqrt(t[0]);
        R.scal[rslot_h(k, k)] = nk;
        R.scal[rslot_h(k, k) + 1] = 0.0;
        R.scal[S_GMRES_F + k] = (double)(float)(nk > 0 ? 1.0 / nk : 0.0);
    });
}
// z += sum_{j<k} c_j basis[j], c_j = scal[S_GCR_C + 2j]
__global__ void __launch_bounds__(kHalfThreads) k_h_multi_axpy(float2* __restrict__ z, const uint2* __restrict__ B,
                                                                const float* __restrict__ S, Geom g, int k,
                                                                const double* __restrict__ scal) {
    __shared__ float c[2 * K_MAX];
    __shared__ float fac[K_MAX];
    for (int j = threadIdx.x; j < 2 * k; j += blockDim.x) c[j] = (float)scal[S_GCR_C + j];
    for (int j = threadIdx.x; j < k && j < K_MAX; j += blockDim.x) fac[j] = inv_norm(scal + S_GMRES_F + j);
    __syncthreads();
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
    const size_t self = (size_t)X * 12 * g.Vb + l, self6 = (size_t)X * 6 * g.Vb + l, V6 = (size_t)6 * g.V;
    cx<float> acc[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = ld<float>(z + self + (size_t)q * g.Vb);
    for (int j = 0; j < k; ++j) {
        cx<float> v[12];
        ld_site_h(B + (size_t)j * V6 + self6, S[(size_t)j * g.V + s] * fac[j], g.Vb, v);
        const cx<float> cj(c[2 * j], c[2 * j + 1]);
#pragma unroll
        for (int q = 0; q < 12; ++q) cmad(acc[q], cj, v[q]);
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) st<float>(z + self + (size_t)q * g.Vb, acc[q]);
}

// ---------------------------------------------------------------- launchers
void links_to_half(uint2* U16, const float2* U32, const Geom& g, cudaStream_t st) {
    const long long n = 4LL * g.Vc * 5 * g.Vb;
    note_launch();
    k_links_to_half<<<(int)std::min<long long>((n + 255) / 256, 16LL * device_sm_count()), 256, 0, st>>>(U16, U32, g);
}
void to_half(HalfSpinor h, const float2* x, const Geom& g, cudaStream_t st) {
    note_launch();
    k_to_half<<<half_grid(g.V), kHalfThreads, 0, st>>>(h.v, h.s, x, g);
}
void from_half(float2* x, ConstHalfSpinor h, const Geom& g, cudaStream_t st) {
    note_launch();
    k_from_half<<<half_grid(g.V), kHalfThreads, 0, st>>>(x, h.v, h.s, g);
}
void dslash_h_plain(HalfSpinor out, ConstHalfSpinor in, const uint2* U16, const Geom& g, double mass, cudaStream_t st,
                    const double* in_norm) {
    note_launch();
    k_dslash_h<HMODE_PLAIN, true><<<half_grid(g.V), kHalfThreads, 0, st>>>(out.v, out.s, in.v, in.s, in_norm, U16,
                                                                          nullptr, g, (float)(4.0 + mass), 0.0,
                                                                          Reduce{});
}
void dslash_h_xmy(HalfSpinor out, const float2* in, const uint2* U16, const float2* src, const Geom& g, double mass,
                  cudaStream_t st) {
    note_launch();
    k_dslash_h<HMODE_XMY, false><<<half_grid(g.V), kHalfThreads, 0, st>>>(out.v, out.s, in, nullptr, nullptr, U16,
                                                                          src, g, (float)(4.0 + mass), 0.0,
                                                                          Reduce{});
}
void dslash_h_mrdot(HalfSpinor out, ConstHalfSpinor in, const uint2* U16, const Geom& g, double mass, double omega,
                    const Reduce& R, cudaStream_t st) {
    note_launch();
    k_dslash_h<HMODE_MRDOT, true><<<half_grid(g.V), kHalfThreads, 0, st>>>(out.v, out.s, in.v, in.s, nullptr, U16,
                                                                          nullptr, g, (float)(4.0 + mass), omega,
                                                                          R);
}
void h_multidot(const uint2* B, const float* S, const Geom& g, int k, const Reduce& R, cudaStream_t st) {
    note_launch();
    // one block per 128 sites, 2 NJ <= 32 float partial sums each: the context
    // sizes the reduction buffer for V / 128 such blocks (reduce_partial_bytes)
    if (k <= 4) k_h_multidot<4><<<half_grid(g.V), kHalfThreads, 0, st>>>(B, S, g, k, R);
    else if (k <= 8) k_h_multidot<8><<<half_grid(g.V), kHalfThreads, 0, st>>>(B, S, g, k, R);
    else k_h_multidot<16><<<half_grid(g.V), kHalfThreads, 0, st>>>(B, S, g, k, R);
}
void h_orth(uint2* B, float* S, const Geom& g, int k, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_h_orth<<<half_grid(g.V), kHalfThreads, 0, st>>>(B, S, g, k, R);
}
void h_multi_axpy(float2* z, const uint2* B, const float* S, const Geom& g, int k, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_h_multi_axpy<<<half_grid(g.V), kHalfThreads, 0, st>>>(z, B, S, g, k, R.scal);
}
void mr_update_h(float2* e, HalfSpinor r, ConstHalfSpinor q, const Geom& g, bool update_r, const Reduce& R,
                 cudaStream_t st) {
    note_launch();
    k_mr_update_h<<<half_grid(g.V), kHalfThreads, 0, st>>>(e, r.v, r.s, q.v, q.s, g, update_r, R.scal);
}

}  // namespace wmg

// Fine-grid kernels: boundary/internal layout conversion, the Wilson-Dirac
// operator of eq. (2) with spin projection, and BLAS-1 / GCR kernels.
#include <atomic>

#include "mg_launch.h"
#include "mg_wilson.cuh"

namespace wmg {

constexpr int kThreads = 256;

static inline int grid_for(size_t n, int threads = kThreads) {
    size_t b = (n + threads - 1) / threads;
    return (int)(b > 0 ? b : 1);
}
static inline int reduce_grid(size_t n) {
    size_t b = (n + kThreads - 1) / kThreads;
    if (b > (size_t)kMaxReduceBlocks) b = kMaxReduceBlocks;
    return (int)(b > 0 ? b : 1);
}

// ================================================================ layouts
template <typename T>
__global__ void k_spinor_to_internal(v2<T>* out, const double2* __restrict__ in, Geom g) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
    long long lex = lex_site(g, X, l);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 v = in[lex * 12 + k];
        v2<T> o; o.x = (T)v.x; o.y = (T)v.y;
        out[((size_t)X * 12 + k) * g.Vb + l] = o;
    }
}
template <typename T>
__global__ void k_spinor_from_internal(double2* out, const v2<T>* __restrict__ in, Geom g) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
    long long lex = lex_site(g, X, l);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        v2<T> v = in[((size_t)X * 12 + k) * g.Vb + l];
        out[lex * 12 + k] = make_double2((double)v.x, (double)v.y);
    }
}
template <typename T>
__global__ void k_links_to_internal(v2<T>* out, const double2* __restrict__ in, Geom g) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
    long long lex = lex_site(g, X, l);
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            double2 v = in[((size_t)mu * g.V + lex) * 9 + e];
            v2<T> o; o.x = (T)v.x; o.y = (T)v.y;
            out[(((size_t)mu * g.Vc + X) * 9 + e) * g.Vb + l] = o;
        }
}
template <typename Tin, typename Tout>
__global__ void k_convert(v2<Tout>* out, const v2<Tin>* __restrict__ in, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        v2<Tin> v = in[i];
        v2<Tout> o; o.x = (Tout)v.x; o.y = (Tout)v.y;
        out[i] = o;
    }
}

template <typename T> void spinor_to_internal(v2<T>* out, const double2* in, const Geom& g, cudaStream_t st) {
    note_launch();
    k_spinor_to_internal<T><<<grid_for(g.V), kThreads, 0, st>>>(out, in, g);
}
template <typename T> void spinor_from_internal(double2* out, const v2<T>* in, const Geom& g, cudaStream_t st) {
    note_launch();
    k_spinor_from_internal<T><<<grid_for(g.V), kThreads, 0, st>>>(out, in, g);
}
template <typename T> void links_to_internal(v2<T>* out, const double2* in, const Geom& g, cudaStream_t st) {
    note_launch();
    k_links_to_internal<T><<<grid_for(g.V), kThreads, 0, st>>>(out, in, g);
}
template <typename Tin, typename Tout> void convert(v2<Tout>* out, const v2<Tin>* in, size_t n, cudaStream_t st) {
    int grid = (int)std::min<size_t>((n + kThreads - 1) / kThreads, (size_t)device_sm_count() * 16);
    note_launch();
    k_convert<Tin, Tout><<<grid > 0 ? grid : 1, kThreads, 0, st>>>(out, in, n);
}

// FP32 links for the dslash: U4[mu][X][j 4][l] = (U[.][2j], U[.][2j+1]) as float4,
// then U8[mu][X][l] = U[.][8] (36 float2 per site in one allocation)
__global__ void k_links_pair(float2* __restrict__ out, const float2* __restrict__ U, Geom g) {
    const long long n = 4LL * g.V;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long ms = i / g.Vb, l = i - ms * g.Vb;   // ms = mu * Vc + X
        const float2* src = U + ms * 9 * g.Vb + l;
        float4* u4 = reinterpret_cast<float4*>(out) + ms * 4 * g.Vb + l;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 a = src[(2 * j) * g.Vb], b = src[(2 * j + 1) * g.Vb];
            u4[(size_t)j * g.Vb] = make_float4(a.x, a.y, b.x, b.y);
        }
        out[(size_t)32 * g.V + ms * g.Vb + l] = src[8 * g.Vb];
    }
}
void links_pair(float2* out, const float2* U32, const Geom& g, cudaStream_t st) {
    note_launch();
    k_links_pair<<<(int)std::min<long long>((4LL * g.V + kThreads - 1) / kThreads, 16LL * device_sm_count()), kThreads, 0, st>>>(out, U32, g);
}

// ================================================================ Wilson operator
template <typename T>
__device__ __forceinline__ void load_spinor(cx<T> (&p)[4][3], const v2<T>* __restrict__ base, int Vb) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) p[s][c] = ldg<T>(base + (3 * s + c) * Vb);
}

// one hop: acc += coef * (1 -/+ gamma_mu) W psi(y), W = U (forward) or U^dag (backward)
template <typename T, int MU, bool FWD>
__device__ __forceinline__ void hop(cx<T> (&acc)[4][3], const v2<T>* __restrict__ in, const v2<T>* __restrict__ U,
                                    const Geom& g, int X, int l, const int (&lc)[4], const int (&xc)[4]) {
    int Xn, ln;
    bool flip;
    neighbour(g, X, l, lc, xc, MU, FWD ? 1 : -1, Xn, ln, flip);
    cx<T> p[4][3];
    load_spinor<T>(p, in + (size_t)Xn * 12 * g.Vb + ln, g.Vb);
    cx<T> h[2][3];
    project<T, MU, FWD>(p, h);
    // link U^mu_x (forward) or U^mu_{x-mu} (backward)
    const size_t ls = FWD ? ((size_t)MU * g.Vc + X) : ((size_t)MU * g.Vc + Xn);
    const int lsite = FWD ? l : ln;
    cx<T> m[9];
    if constexpr (sizeof(T) == 4) {
        // FP32 links in pairs: entries (2j, 2j+1) as one 16-byte word, j < 4, then entry 8
        const float4* u4 = reinterpret_cast<const float4*>(U) + ls * 4 * g.Vb + lsite;
        const float2* u8 = reinterpret_cast<const float2*>(U) + (size_t)32 * g.V + ls * g.Vb + lsite;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 q = __ldg(u4 + (size_t)j * g.Vb);
            m[2 * j] = cx<T>(q.x, q.y);
            m[2 * j + 1] = cx<T>(q.z, q.w);
        }
        const float2 q8 = __ldg(u8);
        m[8] = cx<T>(q8.x, q8.y);
    } else {
        const v2<T>* u = U + ls * 9 * g.Vb + lsite;
#pragma unroll
        for (int e = 0; e < 9; ++e) m[e] = ldg<T>(u + e * g.Vb);
    }
    cx<T> w[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w[0][a] = cx<T>(0, 0);
        w[1][a] = cx<T>(0, 0);
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
    accumulate<T, MU, FWD>(acc, w, flip ? T(0.5) : T(-0.5));
}

// SM count of the current device, looked up once per device (atomic slots)
int device_sm_count() {
    static std::atomic<int> cache[16];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return 152;
    int n = cache[dev].load(std::memory_order_acquire);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cache[dev].store(n, std::memory_order_release);
    }
    return n;
}

// CTA shape of the dslash.  FP32: 128 threads; with 7 CTAs per SM (72
// registers) one thread per site of a 16^3x32 lattice fits one wave of the 152
// SMs (256 threads x 3 CTAs left a 12% second wave: 18.3 -> 14.4 us warm, 28.2
// -> 22.7 us with L2 flushed).  Lattices of several waves take 5 CTAs per SM
// (up to 102 registers: more of each thread's neighbour loads in flight):
// measured on 24^3x64, 99.8 -> 92.2 us with L2 flushed, 93.9 -> 85.8 us back to
// back; 6 gave the same, 8 (64 registers, spills) 111 us.  FP64: 256 x 2.
template <typename T, int MINB> struct DslashShape { static constexpr int threads = 128, blocks = MINB; };
template <int MINB> struct DslashShape<double, MINB> { static constexpr int threads = 256, blocks = 2; };
constexpr int kDslashOneWave = 7, kDslashMultiWave = 5;

template <typename T, int MODE, int MINB>
__global__ void __launch_bounds__(DslashShape<T, MINB>::threads, DslashShape<T, MINB>::blocks)
    k_dslash(v2<T>* __restrict__ out, const v2<T>* __restrict__ in, const v2<T>* __restrict__ U,
             const v2<T>* __restrict__ src, Geom g, T diag, double omega, int slot, Reduce R) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    T red[3] = {0, 0, 0};   // per-site partial sums in T, promoted once for the grid reduction
    if (s < g.V) {
        int X = (int)(s / g.Vb), l = (int)(s - (long long)X * g.Vb);
        int lc[4], xc[4];
        local_coords(g, l, lc);
        coarse_coords(g, X, xc);
        const v2<T>* self = in + (size_t)X * 12 * g.Vb + l;
        cx<T> acc[4][3];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[sp][c] = diag * ldg<T>(self + (3 * sp + c) * g.Vb);
        hop<T, 0, true>(acc, in, U, g, X, l, lc, xc);
        hop<T, 0, false>(acc, in, U, g, X, l, lc, xc);
        hop<T, 1, true>(acc, in, U, g, X, l, lc, xc);
        hop<T, 1, false>(acc, in, U, g, X, l, lc, xc);
        hop<T, 2, true>(acc, in, U, g, X, l, lc, xc);
        hop<T, 2, false>(acc, in, U, g, X, l, lc, xc);
        hop<T, 3, true>(acc, in, U, g, X, l, lc, xc);
        hop<T, 3, false>(acc, in, U, g, X, l, lc, xc);
        v2<T>* o = out + (size_t)X * 12 * g.Vb + l;
        const v2<T>* sr = src + (size_t)X * 12 * g.Vb + l;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                int k = 3 * sp + c;
                cx<T> v = acc[sp][c];
                if (MODE == DS_XMY || MODE == DS_XMY_NORM) v = ld<T>(sr + k * g.Vb) - v;
                st<T>(o + k * g.Vb, v);
                if (MODE == DS_XMY_NORM) red[0] += norm2(v);
                if (MODE == DS_MRDOT) {
                    cx<T> r = ldg<T>(self + k * g.Vb);   // <q, r>: q = D r at this site (cache hit)
                    red[0] += v.r * r.r + v.i * r.i;
                    red[1] += v.r * r.i - v.i * r.r;
                    red[2] += norm2(v);
                }
            }
    }
    if (MODE == DS_XMY_NORM) {
        T v1[1] = {red[0]};
        grid_reduce<1, T>(v1, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) { R.scal[slot] = t[0]; });
    } else if (MODE == DS_MRDOT) {
        T v3[3] = {red[0], red[1], red[2]};
        grid_reduce<3, T>(v3, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[3]) {
            double f = t[2] > 0 ? omega / t[2] : 0.0;
            R.scal[S_MR_ALPHA] = f * t[0];
            R.scal[S_MR_ALPHA + 1] = f * t[1];
        });
    }
}

template <typename T, int MINB>
static void dslash_launch(int mode, v2<T>* out, const v2<T>* in, const v2<T>* U, const v2<T>* src, const Geom& g,
                          T diag, double omega, int slot, const Reduce& R, cudaStream_t st) {
    constexpr int thr = DslashShape<T, MINB>::threads;
    const int grid = grid_for(g.V, thr);
    note_launch();
    switch (mode) {
        case DS_PLAIN: k_dslash<T, DS_PLAIN, MINB><<<grid, thr, 0, st>>>(out, in, U, src, g, diag, omega, slot, R); break;
        case DS_XMY: k_dslash<T, DS_XMY, MINB><<<grid, thr, 0, st>>>(out, in, U, src, g, diag, omega, slot, R); break;
        case DS_XMY_NORM:
            k_dslash<T, DS_XMY_NORM, MINB><<<grid, thr, 0, st>>>(out, in, U, src, g, diag, omega, slot, R);
            break;
        case DS_MRDOT: k_dslash<T, DS_MRDOT, MINB><<<grid, thr, 0, st>>>(out, in, U, src, g, diag, omega, slot, R); break;
    }
}

template <typename T>
void dslash(int mode, v2<T>* out, const v2<T>* in, const v2<T>* U, const v2<T>* src, const Geom& g, double mass,
            double omega, int slot, const Reduce& R, cudaStream_t st) {
    const T diag = (T)(4.0 + mass);
    const long long one_wave = (long long)device_sm_count() * kDslashOneWave * DslashShape<T, kDslashOneWave>::threads;
    if (sizeof(T) == 8 || g.V <= one_wave)
        dslash_launch<T, kDslashOneWave>(mode, out, in, U, src, g, diag, omega, slot, R, st);
    else
        dslash_launch<T, kDslashMultiWave>(mode, out, in, U, src, g, diag, omega, slot, R, st);
}

// ================================================================ BLAS-1
template <typename T> __global__ void k_zero(v2<T>* x, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        v2<T> z; z.x = 0; z.y = 0;
        x[i] = z;
    }
}
template <typename T> __global__ void k_norm2(const v2<T>* __restrict__ x, size_t n, int slot, Reduce R) {
    T a = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a += norm2(ld<T>(x + i));
    T acc[1] = {a};
    grid_reduce<1, T>(acc, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) { R.scal[slot] = t[0]; });
}
template <typename T>
__global__ void k_dot(const v2<T>* __restrict__ x, const v2<T>* __restrict__ y, size_t n, int slot, Reduce R) {
    cx<T> a(0, 0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        cmadc(a, ld<T>(x + i), ld<T>(y + i));
    T acc[2] = {a.r, a.i};
    grid_reduce<2, T>(acc, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[2]) {
        R.scal[slot] = t[0];
        R.scal[slot + 1] = t[1];
    });
}
template <typename T> __global__ void k_scale(v2<T>* x, size_t n, T s) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        st<T>(x + i, s * ld<T>(x + i));
}
template <typename T> __global__ void k_axpy(v2<T>* y, const v2<T>* __restrict__ x, size_t n, T ar, T ai) {
    cx<T> a(ar, ai);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<T> v = ld<T>(y + i);
        cmad(v, a, ld<T>(x + i));
        st<T>(y + i, v);
    }
}
template <typename T>
__global__ void k_mr_update(v2<T>* e, v2<T>* r, const v2<T>* __restrict__ q, size_t n, bool update_r,
                            const double* __restrict__ scal) {
    cx<T> a((T)scal[S_MR_ALPHA], (T)scal[S_MR_ALPHA + 1]);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<T> ri = ld<T>(r + i);
        cx<T> ei = ld<T>(e + i);
        cmad(ei, a, ri);
        st<T>(e + i, ei);
        if (update_r) {
            cx<T> qa = a * ld<T>(q + i);
            st<T>(r + i, ri - qa);
        }
    }
}
template <typename T> __global__ void k_normalize(v2<T>* x, size_t n, const double* __restrict__ scal, int slot) {
    T s = (T)(1.0 / sqrt(scal[slot]));
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        st<T>(x + i, s * ld<T>(x + i));
}

static inline int stream_grid(size_t n) {
    size_t b = (n + kThreads - 1) / kThreads;
    if (b > 16LL * device_sm_count()) b = 16LL * device_sm_count();
    return (int)(b > 0 ? b : 1);
}

template <typename T> void zero(v2<T>* x, size_t n, cudaStream_t st) {
    note_launch();
    k_zero<T><<<stream_grid(n), kThreads, 0, st>>>(x, n);
}
template <typename T> void norm2(const v2<T>* x, size_t n, int slot, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_norm2<T><<<reduce_grid(n), kThreads, 0, st>>>(x, n, slot, R);
}
template <typename T> void dot(const v2<T>* x, const v2<T>* y, size_t n, int slot, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_dot<T><<<reduce_grid(n), kThreads, 0, st>>>(x, y, n, slot, R);
}
template <typename T> void scale(v2<T>* x, size_t n, double s, cudaStream_t st) {
    note_launch();
    k_scale<T><<<stream_grid(n), kThreads, 0, st>>>(x, n, (T)s);
}
template <typename T> void axpy(v2<T>* y, const v2<T>* x, size_t n, double ar, double ai, cudaStream_t st) {
    note_launch();
    k_axpy<T><<<stream_grid(n), kThreads, 0, st>>>(y, x, n, (T)ar, (T)ai);
}
template <typename T>
void mr_update(v2<T>* e, v2<T>* r, const v2<T>* q, size_t n, bool update_r, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_mr_update<T><<<stream_grid(n), kThreads, 0, st>>>(e, r, q, n, update_r, R.scal);
}
template <typename T> void normalize_dev(v2<T>* x, size_t n, int slot, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_normalize<T><<<stream_grid(n), kThreads, 0, st>>>(x, n, R.scal, slot);
}

// ================================================================ GCR
__device__ __forceinline__ int rslot(int j, int k) { return S_GCR_R + 2 * (k * K_MAX + j); }

template <typename T, int NJ>
__global__ void k_gcr_multidot(const v2<T>* __restrict__ basis, size_t n, int k, Reduce R) {
    T a[2 * NJ];
#pragma unroll
    for (int j = 0; j < 2 * NJ; ++j) a[j] = 0;
    const v2<T>* pk = basis + (size_t)k * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<T> v = ld<T>(pk + i);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            if (j < k) {
                cx<T> pj = ld<T>(basis + (size_t)j * n + i);
                cx<T> t(a[2 * j], a[2 * j + 1]);
                cmadc(t, pj, v);
                a[2 * j] = t.r;
                a[2 * j + 1] = t.i;
            }
        }
    }
    grid_reduce<2 * NJ, T>(a, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[2 * NJ]) {
        for (int j = 0; j < k && j < NJ; ++j) {
            R.scal[rslot(j, k)] = t[2 * j];
            R.scal[rslot(j, k) + 1] = t[2 * j + 1];
        }
    });
}
template <typename T>
__global__ void k_gcr_orth_norm(v2<T>* basis, size_t n, int k, Reduce R) {
    __shared__ double beta[2 * K_MAX];
    for (int j = threadIdx.x; j < 2 * k; j += blockDim.x) beta[j] = R.scal[S_GCR_R + 2 * k * K_MAX + j];
    __syncthreads();
    v2<T>* pk = basis + (size_t)k * n;
    T a = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<T> v = ld<T>(pk + i);
        for (int j = 0; j < k; ++j) {
            cx<T> b((T)beta[2 * j], (T)beta[2 * j + 1]);
            cx<T> pj = ld<T>(basis + (size_t)j * n + i);
            v = v - b * pj;
        }
        st<T>(pk + i, v);
        a += norm2(v);
    }
    T acc[1] = {a};
    grid_reduce<1, T>(acc, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) { R.scal[S_GCR_PN2] = t[0]; });
}
template <typename T>
__global__ void k_gcr_cdot(const v2<T>* __restrict__ basis, const v2<T>* __restrict__ r, size_t n, int k, Reduce R) {
    const v2<T>* pk = basis + (size_t)k * n;
    cx<T> a(0, 0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        cmadc(a, ld<T>(pk + i), ld<T>(r + i));
    T acc[2] = {a.r, a.i};
    grid_reduce<2, T>(acc, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[2]) {
        double nk = sqrt(R.scal[S_GCR_PN2]);
        R.scal[rslot(k, k)] = nk;
        R.scal[rslot(k, k) + 1] = 0.0;
        double f = nk > 0 ? 1.0 / nk : 0.0;
        R.scal[S_GCR_C + 2 * k] = t[0] * f;
        R.scal[S_GCR_C + 2 * k + 1] = t[1] * f;
    });
}
template <typename T>
__global__ void k_gcr_update(v2<T>* basis, v2<T>* r, size_t n, int k, Reduce R) {
    double nk = sqrt(R.scal[S_GCR_PN2]);
    T f = (T)(nk > 0 ? 1.0 / nk : 0.0);
    cx<T> c((T)R.scal[S_GCR_C + 2 * k], (T)R.scal[S_GCR_C + 2 * k + 1]);
    v2<T>* pk = basis + (size_t)k * n;
    T a = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<T> p = f * ld<T>(pk + i);
        st<T>(pk + i, p);
        cx<T> v = ld<T>(r + i) - c * p;
        st<T>(r + i, v);
        a += norm2(v);
    }
    T acc[1] = {a};
    grid_reduce<1, T>(acc, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) { R.scal[S_GCR_R2] = t[0]; });
}
template <typename T>
__global__ void k_gcr_xupdate(double2* x, const v2<T>* __restrict__ Z, size_t n, int k, GcrCoef y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<double> v = ld<double>(x + i);
        for (int j = 0; j < k; ++j) {
            v2<T> z = Z[(size_t)j * n + i];
            cx<double> zj((double)z.x, (double)z.y);
            cmad(v, cx<double>(y.c[2 * j], y.c[2 * j + 1]), zj);
        }
        st<double>(x + i, v);
    }
}

template <typename T> void gcr_multidot(const v2<T>* basis, size_t n, int k, const Reduce& R, cudaStream_t st) {
    int grid = reduce_grid(n);
    if (k <= 4) { note_launch(); k_gcr_multidot<T, 4><<<grid, kThreads, 0, st>>>(basis, n, k, R); }
    else if (k <= 8) { note_launch(); k_gcr_multidot<T, 8><<<grid, kThreads, 0, st>>>(basis, n, k, R); }
    else if (k <= 16) { note_launch(); k_gcr_multidot<T, 16><<<grid, kThreads, 0, st>>>(basis, n, k, R); }
    else { note_launch(); k_gcr_multidot<T, 32><<<grid, kThreads, 0, st>>>(basis, n, k, R); }
}
template <typename T> void gcr_orth_norm(v2<T>* basis, size_t n, int k, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_gcr_orth_norm<T><<<reduce_grid(n), kThreads, 0, st>>>(basis, n, k, R);
}
template <typename T>
void gcr_cdot(const v2<T>* basis, const v2<T>* r, size_t n, int k, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_gcr_cdot<T><<<reduce_grid(n), kThreads, 0, st>>>(basis, r, n, k, R);
}
template <typename T> void gcr_update(v2<T>* basis, v2<T>* r, size_t n, int k, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_gcr_update<T><<<reduce_grid(n), kThreads, 0, st>>>(basis, r, n, k, R);
}
template <typename T>
void gcr_xupdate(double2* x, const v2<T>* Z, size_t n, int k, const GcrCoef& y, cudaStream_t st) {
    note_launch();
    k_gcr_xupdate<T><<<stream_grid(n), kThreads, 0, st>>>(x, Z, n, k, y);
}

// ================================================================ GMRES(k) smoother
// One application of GMRES(k) with under-relaxation (Sec. III-IV): Arnoldi
// vectors basis[0..k] (basis[0] = r / beta), column j of the Hessenberg matrix
// Hbar in the scalars: h_ij = scal[rslot(i, j+1)] (i <= j) from
// k_gcr_multidot / k_gcr_orth_norm (one classical Gram-Schmidt pass), and
// h_{j+1,j} = scal[rslot(j+1, j+1)] written when basis[j+1] is normalised.
template <typename T> __global__ void k_gmres_normalize(v2<T>* basis, size_t n, int k, const double* __restrict__ in,
                                                        double* __restrict__ out) {
    const double nk = sqrt(in[S_GCR_PN2]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[rslot(k, k)] = nk;
        out[rslot(k, k) + 1] = 0.0;
    }
    const T f = (T)(nk > 0 ? 1.0 / nk : 0.0);   // a zero vector stays zero (breakdown: exact in the space)
    v2<T>* pk = basis + (size_t)k * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        st<T>(pk + i, f * ld<T>(pk + i));
}
// y = argmin || beta e_1 - Hbar y || by Givens rotations (one thread), then
// scal[S_GCR_C + 2j] = omega y_j.  beta = scal[rslot(0, 0)] (the norm of r,
// recorded when basis[0] was normalised).  The space ends at the first zero
// h_{j+1,j}.
constexpr int kGmresMax = 16;   // largest smoother Krylov dimension (mg_params check)
__global__ void k_gmres_ls(double* scal, int k, double omega) {
    // one warp: lane jj owns column jj of the Hessenberg matrix (lane kGmresMax
    // the right-hand side g), so each Givens rotation is applied to all columns at
    // once with the same arithmetic per column as a serial sweep; the back
    // substitution runs in lane 0 in the usual order
    __shared__ double hr[kGmresMax + 1][kGmresMax + 1], hi[kGmresMax + 1][kGmresMax + 1];
    __shared__ double yr[kGmresMax], yi[kGmresMax];
    __shared__ int s_dim;
    const int lane = threadIdx.x;
    if (blockIdx.x != 0 || lane >= 32 || k > kGmresMax) return;
    // H[i][j] = scal[rslot(i, j + 1)], i <= j + 1; column kGmresMax holds g = beta e_0
    for (int e = lane; e < (kGmresMax + 1) * (kGmresMax + 1); e += 32) {
        const int i = e / (kGmresMax + 1), j = e - i * (kGmresMax + 1);
        double vr = 0.0, vi = 0.0;
        if (j < k && i <= j + 1) {
            const int sl = rslot(i, j + 1);
            vr = scal[sl];
            vi = scal[sl + 1];
        } else if (j == kGmresMax && i == 0) {
            vr = scal[rslot(0, 0)];
        }
        hr[i][j] = vr;
        hi[i][j] = vi;
    }
    __syncwarp();
    if (lane == 0) {
        int dim = k;
        for (int j = 0; j < k; ++j)
            if (!(hr[j + 1][j] > 0)) { dim = j + 1; break; }
        s_dim = dim;
    }
    __syncwarp();
    const int dim = s_dim;
    const int col = lane < dim ? lane : (lane == 31 ? kGmresMax : -1);   // lane 31 carries g
    for (int j = 0; j < dim; ++j) {
        const double ar = hr[j][j], ai = hi[j][j], br = hr[j + 1][j], bi = hi[j + 1][j];
        __syncwarp();
        const double nrm = sqrt(ar * ar + ai * ai + br * br + bi * bi);
        if (nrm > 0 && col >= 0 && (col >= j)) {
            const double cr = ar / nrm, ci = ai / nrm, sr = br / nrm, si = bi / nrm;
            // [conj(c) conj(s); -s c] applied to rows j, j+1
            const double x1r = hr[j][col], x1i = hi[j][col], x2r = hr[j + 1][col], x2i = hi[j + 1][col];
            hr[j][col] = cr * x1r + ci * x1i + sr * x2r + si * x2i;
            hi[j][col] = cr * x1i - ci * x1r + sr * x2i - si * x2r;
            hr[j + 1][col] = -(sr * x1r - si * x1i) + (cr * x2r - ci * x2i);
            hi[j + 1][col] = -(sr * x1i + si * x1r) + (cr * x2i + ci * x2r);
        }
        __syncwarp();
    }
    if (lane == 0) {
        for (int i = dim - 1; i >= 0; --i) {
            double ar = hr[i][kGmresMax], ai = hi[i][kGmresMax];
            for (int jj = i + 1; jj < dim; ++jj) {
                ar -= hr[i][jj] * yr[jj] - hi[i][jj] * yi[jj];
                ai -= hr[i][jj] * yi[jj] + hi[i][jj] * yr[jj];
            }
            const double dr = hr[i][i], di = hi[i][i], dd = dr * dr + di * di;
            yr[i] = dd > 0 ? (ar * dr + ai * di) / dd : 0.0;
            yi[i] = dd > 0 ? (ai * dr - ar * di) / dd : 0.0;
        }
    }
    __syncwarp();
    for (int j = lane; j < k; j += 32) {
        scal[S_GCR_C + 2 * j] = j < dim ? omega * yr[j] : 0.0;
        scal[S_GCR_C + 2 * j + 1] = j < dim ? omega * yi[j] : 0.0;
    }
}
// z += sum_{j<k} c_j basis[j], c_j = scal[S_GCR_C + 2j]
template <typename T>
__global__ void k_multi_axpy(v2<T>* z, const v2<T>* __restrict__ basis, size_t n, int k, const double* __restrict__ scal) {
    __shared__ double c[2 * K_MAX];
    for (int j = threadIdx.x; j < 2 * k; j += blockDim.x) c[j] = scal[S_GCR_C + j];
    __syncthreads();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<T> v = ld<T>(z + i);
        for (int j = 0; j < k; ++j) cmad(v, cx<T>((T)c[2 * j], (T)c[2 * j + 1]), ld<T>(basis + (size_t)j * n + i));
        st<T>(z + i, v);
    }
}
template <typename T> void gmres_normalize(v2<T>* basis, size_t n, int k, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_gmres_normalize<T><<<stream_grid(n), kThreads, 0, st>>>(basis, n, k, R.scal, R.scal);
}
void gmres_ls(const Reduce& R, int k, double omega, cudaStream_t st) {
    note_launch();
    k_gmres_ls<<<1, 32, 0, st>>>(R.scal, k, omega);
}
template <typename T> void multi_axpy(v2<T>* z, const v2<T>* basis, size_t n, int k, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_multi_axpy<T><<<stream_grid(n), kThreads, 0, st>>>(z, basis, n, k, R.scal);
}

// ================================================================ instantiations
#define INST(T)                                                                                                     \
    template void spinor_to_internal<T>(v2<T>*, const double2*, const Geom&, cudaStream_t);                         \
    template void spinor_from_internal<T>(double2*, const v2<T>*, const Geom&, cudaStream_t);                       \
    template void links_to_internal<T>(v2<T>*, const double2*, const Geom&, cudaStream_t);                          \
    template void dslash<T>(int, v2<T>*, const v2<T>*, const v2<T>*, const v2<T>*, const Geom&, double, double, int, \
                            const Reduce&, cudaStream_t);                                                           \
    template void zero<T>(v2<T>*, size_t, cudaStream_t);                                                            \
    template void norm2<T>(const v2<T>*, size_t, int, const Reduce&, cudaStream_t);                                 \
    template void dot<T>(const v2<T>*, const v2<T>*, size_t, int, const Reduce&, cudaStream_t);                     \
    template void scale<T>(v2<T>*, size_t, double, cudaStream_t);                                                   \
    template void axpy<T>(v2<T>*, const v2<T>*, size_t, double, double, cudaStream_t);                              \
    template void mr_update<T>(v2<T>*, v2<T>*, const v2<T>*, size_t, bool, const Reduce&, cudaStream_t);            \
    template void normalize_dev<T>(v2<T>*, size_t, int, const Reduce&, cudaStream_t);                               \
    template void gcr_multidot<T>(const v2<T>*, size_t, int, const Reduce&, cudaStream_t);                          \
    template void gcr_orth_norm<T>(v2<T>*, size_t, int, const Reduce&, cudaStream_t);                               \
    template void gcr_cdot<T>(const v2<T>*, const v2<T>*, size_t, int, const Reduce&, cudaStream_t);                \
    template void gcr_update<T>(v2<T>*, v2<T>*, size_t, int, const Reduce&, cudaStream_t);                          \
    template void gcr_xupdate<T>(double2*, const v2<T>*, size_t, int, const GcrCoef&, cudaStream_t);          \
    template void gmres_normalize<T>(v2<T>*, size_t, int, const Reduce&, cudaStream_t);                        \
    template void multi_axpy<T>(v2<T>*, const v2<T>*, size_t, int, const Reduce&, cudaStream_t);
INST(float)
INST(double)
#undef INST
template void convert<double, float>(v2<float>*, const v2<double>*, size_t, cudaStream_t);
template void convert<float, double>(v2<double>*, const v2<float>*, size_t, cudaStream_t);
template void convert<double, double>(v2<double>*, const v2<double>*, size_t, cudaStream_t);
template void convert<float, float>(v2<float>*, const v2<float>*, size_t, cudaStream_t);

}  // namespace wmg

// Shared device-side definitions of the Wilson-Dirac multigrid library.
//
// Internal data layout ("aggregate-major SoA"): fine sites are ordered block
// by block, s = X * Vb + l, with X the lexicographic index of the aggregate
// (coarse site) and l the lexicographic index inside the Vb = B0*B1*B2*B3
// sites of the block.  Per-site components are stored component-major inside
// each block, so a warp of consecutive l reads consecutive addresses:
//   fine spinor   T2 v[X][k 12][l]          k = spin*3 + colour
//   links         T2 U[mu][X][e 9][l]       e = row*3 + col
//   prolongator   T2 P[X][s 2][i Nv][k 6][l] k = spin-in-chirality*3 + colour
//   coarse vector T2 y[X][a 2Nv]
//   coarse op     T2 A[X][d 9][b][a]        column-major 2Nv x 2Nv blocks
// This makes restriction, prolongation, block orthonormalisation and the
// coarse-operator build contiguous per aggregate, and keeps dslash loads
// coalesced.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wmg {

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T> using v2 = typename vec2<T>::type;

// complex number in registers
template <typename T> struct cx {
    T r, i;
    __host__ __device__ cx() {}
    __host__ __device__ cx(T a, T b) : r(a), i(b) {}
};
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return cx<T>(a.r + b.r, a.i + b.i); }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return cx<T>(a.r - b.r, a.i - b.i); }
template <typename T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return cx<T>(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <typename T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return cx<T>(s * a.r, s * a.i); }
template <typename T> __device__ __forceinline__ cx<T> conj(cx<T> a) { return cx<T>(a.r, -a.i); }
template <typename T> __device__ __forceinline__ cx<T> mul_i(cx<T> a) { return cx<T>(-a.i, a.r); }     // i a
template <typename T> __device__ __forceinline__ cx<T> mul_mi(cx<T> a) { return cx<T>(a.i, -a.r); }    // -i a
// a += b * c
template <typename T> __device__ __forceinline__ void cmad(cx<T>& a, cx<T> b, cx<T> c) {
    a.r = fma(b.r, c.r, a.r); a.r = fma(-b.i, c.i, a.r);
    a.i = fma(b.r, c.i, a.i); a.i = fma(b.i, c.r, a.i);
}
// a += conj(b) * c
template <typename T> __device__ __forceinline__ void cmadc(cx<T>& a, cx<T> b, cx<T> c) {
    a.r = fma(b.r, c.r, a.r); a.r = fma(b.i, c.i, a.r);
    a.i = fma(b.r, c.i, a.i); a.i = fma(-b.i, c.r, a.i);
}
template <typename T> __device__ __forceinline__ T norm2(cx<T> a) { return a.r * a.r + a.i * a.i; }

template <typename T> __device__ __forceinline__ cx<T> ld(const v2<T>* p) { v2<T> v = *p; return cx<T>(v.x, v.y); }
template <typename T> __device__ __forceinline__ cx<T> ldg(const v2<T>* p) { v2<T> v = __ldg(p); return cx<T>(v.x, v.y); }
template <typename T> __device__ __forceinline__ void st(v2<T>* p, cx<T> a) { v2<T> v; v.x = a.r; v.y = a.i; *p = v; }

// lattice geometry, passed by value to kernels
struct Geom {
    int L[4], B[4], Lc[4];
    int lstride[4];   // stride of local coordinate mu inside a block
    int xstride[4];   // stride of coarse coordinate mu
    int Vb;           // sites per block
    int Vc;           // blocks (coarse sites)
    long long V;      // fine sites
    int tap;          // antiperiodic in t
};

__host__ __device__ inline void local_coords(const Geom& g, int l, int lc[4]) {
    lc[0] = l % g.B[0]; l /= g.B[0];
    lc[1] = l % g.B[1]; l /= g.B[1];
    lc[2] = l % g.B[2];
    lc[3] = l / g.B[2];
}
__host__ __device__ inline void coarse_coords(const Geom& g, int X, int xc[4]) {
    xc[0] = X % g.Lc[0]; X /= g.Lc[0];
    xc[1] = X % g.Lc[1]; X /= g.Lc[1];
    xc[2] = X % g.Lc[2];
    xc[3] = X / g.Lc[2];
}
// lexicographic (boundary) site index of internal (X, l)
__host__ __device__ inline long long lex_site(const Geom& g, int X, int l) {
    int lc[4], xc[4];
    local_coords(g, l, lc);
    coarse_coords(g, X, xc);
    long long c0 = xc[0] * g.B[0] + lc[0], c1 = xc[1] * g.B[1] + lc[1];
    long long c2 = xc[2] * g.B[2] + lc[2], c3 = xc[3] * g.B[3] + lc[3];
    return c0 + (long long)g.L[0] * (c1 + (long long)g.L[1] * (c2 + (long long)g.L[2] * c3));
}

// neighbour (Xn, ln) of site (X, l) in direction mu, dir = +1/-1; flip = crossing
// of the antiperiodic t face
__device__ __forceinline__ void neighbour(const Geom& g, int X, int l, const int lc[4], const int xc[4], int mu,
                                          int dir, int& Xn, int& ln, bool& flip) {
    int lm = lc[mu] + dir;
    flip = false;
    Xn = X;
    if (lm >= 0 && lm < g.B[mu]) {
        ln = l + dir * g.lstride[mu];
    } else {
        ln = l - dir * (g.B[mu] - 1) * g.lstride[mu];
        int xm = xc[mu] + dir;
        if (xm >= g.Lc[mu]) { Xn = X - (g.Lc[mu] - 1) * g.xstride[mu]; flip = (mu == 3) && g.tap; }
        else if (xm < 0) { Xn = X + (g.Lc[mu] - 1) * g.xstride[mu]; flip = (mu == 3) && g.tap; }
        else Xn = X + dir * g.xstride[mu];
    }
}
// coarse neighbour for stencil slot d (0: self, 1+2mu: +mu, 2+2mu: -mu), periodic
__device__ __forceinline__ int coarse_neighbour(const Geom& g, int X, int d) {
    if (d == 0) return X;
    int mu = (d - 1) >> 1;
    int dir = (d & 1) ? 1 : -1;
    int xc[4];
    coarse_coords(g, X, xc);
    int xm = xc[mu] + dir;
    if (xm >= g.Lc[mu]) return X - (g.Lc[mu] - 1) * g.xstride[mu];
    if (xm < 0) return X + (g.Lc[mu] - 1) * g.xstride[mu];
    return X + dir * g.xstride[mu];
}

// ---------------------------------------------------------------- scalars
// Device-resident scalars of the solvers (one double array per context).
enum ScalarSlot {
    S_MR_ALPHA = 0,      // 2: omega <q,r>/<q,q>
    S_NORM_A = 2,        // generic norm^2 results
    S_NORM_B = 3,
    S_DOT = 4,           // 2: generic dot
    S_CG_ALPHA = 8,
    S_CG_BETA = 9,
    S_CG_GAMMA = 10,
    S_CG_RC2 = 11,       // ||r_c||^2 at start
    S_CG_R2 = 12,        // current ||r||^2
    S_CG_ITERS = 13,
    S_CG_DONE = 14,
    S_CG_TOL2 = 15,
    S_CG_MAXIT = 16,
    S_CG_TOTAL = 17,     // coarse iterations accumulated over a solve
    S_GCR_PN2 = 20,      // ||p_k||^2 after orthogonalisation
    S_GCR_R2 = 21,       // ||r||^2 after the update
    S_GMRES_F = 24,      // 17: 1 / ||v_k|| of the FP16 Arnoldi basis, rounded to float
    S_EO = 42,           // 12: red-black CG (gamma x2, |q|^2, |r|^2, tol^2, done, iterations, residual norms)
    S_GCR_R = 64,        // R[j][k] complex, K_MAX x K_MAX (column k, row j): 2*K_MAX*K_MAX
    S_GCR_C = 64 + 2 * 32 * 32,   // c_k complex
    S_COUNT = 64 + 2 * 32 * 32 + 64
};
constexpr int K_MAX = 32;

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-reduce N doubles; result valid in thread 0.  Needs blockDim.x % 32 == 0,
// blockDim.x <= 1024.  Fixed summation order for a fixed blockDim.
template <int N>
__device__ __forceinline__ void block_reduce(double (&v)[N], double (*sh)[32]) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double x = lane < nw ? sh[k][lane] : 0.0;
            v[k] = warp_sum(x);
        }
    }
}

template <typename TA> __device__ __forceinline__ TA warp_sum_acc(TA v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Block-reduce N values of type TA; result valid in thread 0.
template <int N, typename TA>
__device__ __forceinline__ void block_reduce_acc(TA (&v)[N], TA (*sh)[32]) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum_acc(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            TA x = lane < nw ? sh[k][lane] : TA(0);
            v[k] = warp_sum_acc(x);
        }
    }
}

// Smallest partial-sum buffer of the grid reductions (Reduce::partials); a
// context sizes its own for its lattice (reduce_partial_bytes).
constexpr int kMaxReduceBlocks = 1216;   // 152 SMs x 8
constexpr size_t kReducePartialsBytes = (size_t)kMaxReduceBlocks * 64 * sizeof(double);

// Single-pass deterministic grid reduction: every block writes its partial
// sums, the last block to arrive adds them in block order and calls
// fin(total) on thread 0 (totals promoted to double).  TA is the accumulation
// type inside blocks (float for the FP32 path: the FP64 pipe of this part is
// narrow).  `partials` holds `cap` bytes, `ticket` is one zeroed counter (reset
// to 0 by the last block).  A grid whose partials would not fit writes
// nothing and reports NaN totals (a launcher bug made visible, not memory
// written out of bounds).
template <int N, typename TA = double, typename Fin>
__device__ __forceinline__ void grid_reduce(TA (&v)[N], double* partials, unsigned int* ticket, size_t cap, Fin fin) {
    if ((size_t)gridDim.x * N * sizeof(TA) > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double t[N];
#pragma unroll
            for (int k = 0; k < N; ++k) t[k] = __longlong_as_double(0x7ff8000000000000LL);
            fin(t);
        }
        return;
    }
    __shared__ TA sh[N][32];
    __shared__ bool is_last;
    block_reduce_acc<N, TA>(v, sh);
    TA* part = reinterpret_cast<TA*>(partials);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) part[(size_t)blockIdx.x * N + k] = v[k];
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    TA acc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] = TA(0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < N; ++k) acc[k] += __ldcg(part + (size_t)b * N + k);
    }
    block_reduce_acc<N, TA>(acc, sh);
    if (threadIdx.x == 0) {
        double t[N];
#pragma unroll
        for (int k = 0; k < N; ++k) t[k] = (double)acc[k];
        fin(t);
        *ticket = 0u;
    }
}

}  // namespace wmg

// Transfer and coarse-level kernels: block orthonormalisation of the
// prototypes (eq. 4 with the chirality split), restriction r_c = P^dag r,
// prolongation e = P y, the Galerkin coarse operator D_c = P^dag D P and its
// nearest-neighbour application, and the CGNR (CGLS) coarse solve steps.
#include <atomic>
#include "mg_launch.h"
#include "mg_sync.cuh"

namespace wmg {

constexpr int kThreads = 256;

static inline int reduce_grid(size_t n) {
    size_t b = (n + kThreads - 1) / kThreads;
    if (b > (size_t)kMaxReduceBlocks) b = kMaxReduceBlocks;
    return (int)(b > 0 ? b : 1);
}

// ================================================================ block orthonormalisation
// One CTA per (aggregate X, chirality s).  Column i of the panel is prototype i
// restricted to X and to the spins of s (6*Vb complex).  Gram-Schmidt applied
// twice in index order with all projections of a pass at once (classical form:
// c = Q_<i^dag w, w -= Q_<i c), then normalisation: the unique Q factor with a
// positive real R-diagonal, the same as modified Gram-Schmidt twice up to
// rounding.  The column being orthogonalised sits in shared memory; warp w
// forms the projections on columns w, w + 8, ... with warp shuffles, so a
// pass costs three CTA barriers instead of one block reduction per column.
constexpr int kOrthoMaxNv = 64;   // nvec <= 25 (parameter check)

__device__ __forceinline__ double block_sum(double v, double* sh) {
    double a[1] = {v};
    block_reduce<1>(a, (double (*)[32])sh);
    __syncthreads();
    if (threadIdx.x == 0) sh[32] = a[0];
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) k_block_ortho(double2* __restrict__ P, const double2* __restrict__ Vin, int nv,
                                                     Geom g, int* status) {
    extern __shared__ double2 wsh[];            // the column being orthogonalised, 6 * Vb entries
    __shared__ double sh[2 * 32 + 2];
    __shared__ double2 cj[kOrthoMaxNv];        // projections of the current pass
    const int X = blockIdx.x >> 1, s = blockIdx.x & 1;
    const int len = 6 * g.Vb, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t vstride = (size_t)g.Vc * 12 * g.Vb;       // one prototype
    double2* panel = P + ((size_t)X * 2 + s) * nv * len;
    for (int i = 0; i < nv; ++i) {
        const double2* vi = Vin + (size_t)i * vstride + ((size_t)X * 12 + 6 * s) * g.Vb;   // k = 6s..6s+5 contiguous
        double n0 = 0;
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            const double2 v = vi[e];
            wsh[e] = v;
            n0 += v.x * v.x + v.y * v.y;
        }
        n0 = block_sum(n0, sh);   // its barriers also publish wsh
        for (int pass = 0; pass < 2 && i > 0; ++pass) {
            // c_j = <q_j, w>, j < i: one warp per column, lanes over the entries
            for (int j = warp; j < i; j += nw) {
                const double2* qj = panel + (size_t)j * len;
                cx<double> c(0, 0);
                for (int e = lane; e < len; e += 32) cmadc(c, ld<double>(qj + e), ld<double>(wsh + e));
                c.r = warp_sum(c.r);
                c.i = warp_sum(c.i);
                if (lane == 0) cj[j] = make_double2(c.r, c.i);
            }
            __syncthreads();
            // w -= sum_j c_j q_j
            for (int e = threadIdx.x; e < len; e += blockDim.x) {
                cx<double> w = ld<double>(wsh + e);
                for (int j = 0; j < i; ++j) w = w - cx<double>(cj[j].x, cj[j].y) * ld<double>(panel + (size_t)j * len + e);
                st<double>(wsh + e, w);
            }
            __syncthreads();
        }
        double n = 0;
        for (int e = threadIdx.x; e < len; e += blockDim.x) n += norm2(ld<double>(wsh + e));
        n = sqrt(block_sum(n, sh));
        if (!(n > 1e-12 * sqrt(n0))) {
            if (threadIdx.x == 0) atomicExch(status, 1);
            n = 1.0;
        }
        const double f = 1.0 / n;
        double2* qi = panel + (size_t)i * len;
        for (int e = threadIdx.x; e < len; e += blockDim.x) st<double>(qi + e, f * ld<double>(wsh + e));
        __syncthreads();   // column i visible to the block before it is re-read
    }
}

void block_orthonormalize(double2* P, const double2* V, int nv, const Geom& g, int* d_status, cudaStream_t st) {
    const size_t sm = sizeof(double2) * 6 * g.Vb;   // <= 32.7 KB: blocks hold at most 341 sites (parameter check)
    note_launch();
    k_block_ortho<<<2 * g.Vc, kThreads, sm, st>>>(P, V, nv, g, d_status);
}

// ================================================================ restriction / prolongation
// r_c[X][s*Nv + i] = <P_(X,s,i), r>: one CTA per (X, s); the chirality-s half of
// r on X (6*Vb contiguous) is staged in shared memory, warp w handles i = w, w+8, ...
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(v2<T>* __restrict__ rc, const v2<T>* __restrict__ P,
                                                  const v2<T>* __restrict__ r, int nv, Geom g, int cstride, int coff) {
    extern __shared__ unsigned char smem_raw[];
    v2<T>* rs = reinterpret_cast<v2<T>*>(smem_raw);
    int X = blockIdx.x >> 1, s = blockIdx.x & 1;
    int len = 6 * g.Vb;
    const v2<T>* rX = r + ((size_t)X * 12 + 6 * s) * g.Vb;
    for (int e = threadIdx.x; e < len; e += blockDim.x) rs[e] = rX[e];
    __syncthreads();
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const v2<T>* panel = P + ((size_t)X * 2 + s) * nv * len;
    for (int i = warp; i < nv; i += nw) {
        const v2<T>* pi = panel + (size_t)i * len;
        cx<T> a(0, 0);
        for (int e = lane; e < len; e += 32) cmadc(a, ldg<T>(pi + e), ld<T>(rs + e));
        double ar = warp_sum((double)a.r), ai = warp_sum((double)a.i);
        if (lane == 0) {
            v2<T> o; o.x = (T)ar; o.y = (T)ai;
            rc[((size_t)X * 2 * nv + s * nv + i) * cstride + coff] = o;
        }
    }
}
// e[X][k][l] = sum_i P[X][s(k)][i][k%6][l] y[X][s(k)*Nv + i]
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(v2<T>* __restrict__ e, const v2<T>* __restrict__ P,
                                                 const v2<T>* __restrict__ yc, int nv, Geom g, int cstride, int coff) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;   // over V*12 as (X, k, l)
    long long total = g.V * 12;
    if (idx >= total) return;
    int l = (int)(idx % g.Vb);
    long long t = idx / g.Vb;
    int k = (int)(t % 12);
    int X = (int)(t / 12);
    int s = k / 6, kk = k - 6 * s;
    int len = 6 * g.Vb;
    const v2<T>* p = P + (((size_t)X * 2 + s) * nv * 6 + kk) * g.Vb + l;
    const v2<T>* y = yc + ((size_t)X * 2 * nv + s * nv) * cstride + coff;
    cx<T> a(0, 0);
    for (int i = 0; i < nv; ++i) cmad(a, ldg<T>(p + (size_t)i * len), ldg<T>(y + (size_t)i * cstride));
    st<T>(e + idx, a);
}

template <typename T>
void restrict_(v2<T>* rc, const v2<T>* P, const v2<T>* r, int nv, const Geom& g, cudaStream_t st, int cstride, int coff) {
    size_t sm = sizeof(v2<T>) * 6 * g.Vb;
    note_launch();
    k_restrict<T><<<2 * g.Vc, kThreads, sm, st>>>(rc, P, r, nv, g, cstride, coff);
}
template <typename T>
void prolong(v2<T>* e, const v2<T>* P, const v2<T>* yc, int nv, const Geom& g, cudaStream_t st, int cstride, int coff) {
    long long total = g.V * 12;
    note_launch();
    k_prolong<T><<<(int)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(e, P, yc, nv, g, cstride, coff);
}

// ================================================================ coarse operator build
// One CTA per (aggregate X, hop h = 2*mu + (0 fwd | 1 bwd)).  For site chunks
// of X it forms W_b(x) = H_h(x) P_b(y) for every coarse column b (H_h the
// hop of eq. 2 from x to y = x +/- mu, P_b column b at y) and accumulates
// conj(P_a(x)) . W_b(x) over the 6 components of chirality s_a.  Hops leaving
// X through its face in direction h go to A[X][1+h]; hops staying inside X go
// to Aself[X][h] (summed later with the diagonal (4+m)).  FP64 throughout.
constexpr int kBuildChunk = 8;
// stride (complex entries) of one (site, column) spinor in the build's shared
// memory: 13, not 12, so the lanes of a warp (consecutive columns) fall on
// distinct banks in the product loop (12 put every fourth lane on one bank)
constexpr int kWStride = 13;

template <typename TC, int MU, bool FWD>
__device__ __forceinline__ void hop_column(const cx<TC> (&p)[4][3], const v2<TC>* __restrict__ u, int Vb, TC coef,
                                           cx<TC> (&out)[4][3]) {
    // spin projection (same convention as the fine operator)
    cx<TC> h[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 0) {
            h[0][c] = FWD ? p[0][c] + mul_mi(p[3][c]) : p[0][c] + mul_i(p[3][c]);
            h[1][c] = FWD ? p[1][c] + mul_mi(p[2][c]) : p[1][c] + mul_i(p[2][c]);
        } else if (MU == 1) {
            h[0][c] = FWD ? p[0][c] + p[3][c] : p[0][c] - p[3][c];
            h[1][c] = FWD ? p[1][c] - p[2][c] : p[1][c] + p[2][c];
        } else if (MU == 2) {
            h[0][c] = FWD ? p[0][c] + mul_mi(p[2][c]) : p[0][c] + mul_i(p[2][c]);
            h[1][c] = FWD ? p[1][c] + mul_i(p[3][c]) : p[1][c] + mul_mi(p[3][c]);
        } else {
            h[0][c] = FWD ? p[0][c] - p[2][c] : p[0][c] + p[2][c];
            h[1][c] = FWD ? p[1][c] - p[3][c] : p[1][c] + p[3][c];
        }
    }
    cx<TC> w[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w[0][a] = cx<TC>(0, 0);
        w[1][a] = cx<TC>(0, 0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (FWD) {
                cx<TC> uab = ld<TC>(u + (3 * a + b) * Vb);
                cmad(w[0][a], uab, h[0][b]);
                cmad(w[1][a], uab, h[1][b]);
            } else {
                cx<TC> uba = ld<TC>(u + (3 * b + a) * Vb);
                cmadc(w[0][a], uba, h[0][b]);
                cmadc(w[1][a], uba, h[1][b]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<TC> w0 = coef * w[0][c], w1 = coef * w[1][c];
        out[0][c] = w0;
        out[1][c] = w1;
        if (MU == 0) { out[2][c] = FWD ? mul_i(w1) : mul_mi(w1); out[3][c] = FWD ? mul_i(w0) : mul_mi(w0); }
        else if (MU == 1) { out[2][c] = FWD ? cx<TC>(-w1.r, -w1.i) : w1; out[3][c] = FWD ? w0 : cx<TC>(-w0.r, -w0.i); }
        else if (MU == 2) { out[2][c] = FWD ? mul_i(w0) : mul_mi(w0); out[3][c] = FWD ? mul_mi(w1) : mul_i(w1); }
        else { out[2][c] = FWD ? cx<TC>(-w0.r, -w0.i) : w0; out[3][c] = FWD ? cx<TC>(-w1.r, -w1.i) : w1; }
    }
}

// TC: precision of the products (double, or float with FP64 accumulation of
// the per-chunk sums).
template <typename TC, int MU, bool FWD>
__device__ void build_hop(double2* __restrict__ A, double2* __restrict__ Aself, const v2<TC>* __restrict__ P,
                          const v2<TC>* __restrict__ U, int nv, const Geom& g, int X, int h, v2<TC>* Wsh,
                          v2<TC>* Psh, unsigned char* leaves) {
    const int nc = 2 * nv, len = 6 * g.Vb;
    const int npair = nc * nc;
    constexpr int kMaxPairs = 10;                      // nc <= 50 with 256 threads
    cx<double> acc_out[kMaxPairs], acc_in[kMaxPairs];
#pragma unroll
    for (int q = 0; q < kMaxPairs; ++q) { acc_out[q] = cx<double>(0, 0); acc_in[q] = cx<double>(0, 0); }
    int xcX[4];
    coarse_coords(g, X, xcX);
    for (int l0 = 0; l0 < g.Vb; l0 += kBuildChunk) {
        int cs = min(kBuildChunk, g.Vb - l0);
        // W_b(x) for x in chunk, all columns b: Wsh[(xi*nc + b)*kWStride + k]
        for (int t = threadIdx.x; t < cs * nc; t += blockDim.x) {
            int xi = t / nc, b = t - xi * nc;
            int l = l0 + xi;
            int lc[4];
            local_coords(g, l, lc);
            int Xn, ln;
            bool flip;
            neighbour(g, X, l, lc, xcX, MU, FWD ? 1 : -1, Xn, ln, flip);
            if (b == 0) leaves[xi] = (FWD ? lc[MU] == g.B[MU] - 1 : lc[MU] == 0) ? 1 : 0;
            int sb = b / nv, ib = b - sb * nv;
            cx<TC> p[4][3];
            const v2<TC>* col = P + (((size_t)Xn * 2 + sb) * nv + ib) * len;
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    int s_sp = sp >> 1;
                    p[sp][c] = (s_sp == sb) ? ld<TC>(col + ((sp & 1) * 3 + c) * g.Vb + ln) : cx<TC>(0, 0);
                }
            const v2<TC>* u = FWD ? U + ((size_t)MU * g.Vc + X) * 9 * g.Vb + l : U + ((size_t)MU * g.Vc + Xn) * 9 * g.Vb + ln;
            cx<TC> o[4][3];
            hop_column<TC, MU, FWD>(p, u, g.Vb, flip ? TC(0.5) : TC(-0.5), o);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) st<TC>(Wsh + ((size_t)xi * nc + b) * kWStride + 3 * sp + c, o[sp][c]);
        }
        // P_a(x) for x in chunk: Psh[(xi*nc + a)*6 + kk]
        for (int t = threadIdx.x; t < cs * nc * 6; t += blockDim.x) {
            int kk = t % 6, r = t / 6;
            int a = r % nc, xi = r / nc;
            int sa = a / nv, ia = a - sa * nv;
            Psh[t] = P[(((size_t)X * 2 + sa) * nv + ia) * len + kk * g.Vb + l0 + xi];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kMaxPairs; ++q) {
            int pr = threadIdx.x + q * blockDim.x;
            if (pr < npair) {
                int a = pr / nc, b = pr - a * nc;
                int sa = a / nv;
                cx<TC> co(0, 0), ci(0, 0);
                for (int xi = 0; xi < cs; ++xi) {
                    cx<TC> t(0, 0);
#pragma unroll
                    for (int kk = 0; kk < 6; ++kk)
                        cmadc(t, ld<TC>(Psh + ((size_t)xi * nc + a) * 6 + kk),
                              ld<TC>(Wsh + ((size_t)xi * nc + b) * kWStride + 6 * sa + kk));
                    if (leaves[xi]) co = co + t;
                    else ci = ci + t;
                }
                acc_out[q] = acc_out[q] + cx<double>((double)co.r, (double)co.i);
                acc_in[q] = acc_in[q] + cx<double>((double)ci.r, (double)ci.i);
            }
        }
        __syncthreads();
    }
    // column-major output: A[X][d][b][a]
#pragma unroll
    for (int q = 0; q < kMaxPairs; ++q) {
        int pr = threadIdx.x + q * blockDim.x;
        if (pr < npair) {
            int a = pr / nc, b = pr - a * nc;
            st<double>(A + (((size_t)X * 9 + 1 + h) * nc + b) * nc + a, acc_out[q]);
            st<double>(Aself + (((size_t)X * 8 + h) * nc + b) * nc + a, acc_in[q]);
        }
    }
}

template <typename TC>
__global__ void __launch_bounds__(256) k_coarse_hop(double2* A, double2* Aself, const v2<TC>* __restrict__ P,
                                                    const v2<TC>* __restrict__ U, int nv, Geom g) {
    extern __shared__ unsigned char smem_raw[];
    const int nc = 2 * nv;
    v2<TC>* Wsh = reinterpret_cast<v2<TC>*>(smem_raw);
    v2<TC>* Psh = Wsh + (size_t)kBuildChunk * nc * kWStride;
    unsigned char* leaves = reinterpret_cast<unsigned char*>(Psh + (size_t)kBuildChunk * nc * 6);
    int X = blockIdx.x >> 3, h = blockIdx.x & 7;
    switch (h) {
        case 0: build_hop<TC, 0, true>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 1: build_hop<TC, 0, false>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 2: build_hop<TC, 1, true>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 3: build_hop<TC, 1, false>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 4: build_hop<TC, 2, true>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 5: build_hop<TC, 2, false>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 6: build_hop<TC, 3, true>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        default: build_hop<TC, 3, false>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
    }
}
// A[X][0] = (4+m) I + sum_h Aself[X][h] (fixed order)
__global__ void k_coarse_diag(double2* A, const double2* __restrict__ Aself, int nc, double diag, Geom g) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)g.Vc * nc * nc;
    if (idx >= total) return;
    int X = (int)(idx / (nc * nc));
    int r = (int)(idx - (long long)X * nc * nc);    // b*nc + a
    int b = r / nc, a = r - b * nc;
    cx<double> v(a == b ? diag : 0.0, 0.0);
    for (int h = 0; h < 8; ++h) v = v + ld<double>(Aself + ((size_t)X * 8 + h) * nc * nc + r);
    st<double>(A + (size_t)X * 9 * nc * nc + r, v);
}

template <typename TC>
void coarse_build_t(double2* A, double2* Aself, const v2<TC>* P, const v2<TC>* U, int nv, double mass, const Geom& g,
                    cudaStream_t st) {
    int nc = 2 * nv;
    size_t sm = sizeof(v2<TC>) * kBuildChunk * nc * (kWStride + 6) + kBuildChunk + 16;
    cudaFuncSetAttribute(k_coarse_hop<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    note_launch();
    k_coarse_hop<TC><<<g.Vc * 8, kThreads, sm, st>>>(A, Aself, P, U, nv, g);
    long long total = (long long)g.Vc * nc * nc;
    note_launch();
    k_coarse_diag<<<(int)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(A, Aself, nc, 4.0 + mass, g);
}
void coarse_build_f32(double2* A, double2* Aself, const float2* P, const float2* U, int nv, double mass, const Geom& g,
                      cudaStream_t st) {
    coarse_build_t<float>(A, Aself, P, U, nv, mass, g, st);
}

void coarse_build(double2* A, double2* Aself, const double2* P, const double2* U, int nv, double mass, const Geom& g,
                  cudaStream_t st) {
    coarse_build_t<double>(A, Aself, P, U, nv, mass, g, st);
}

__global__ void k_coarse_shift(double2* A, int nc, double dm, int Vc) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)Vc * nc) return;
    int X = (int)(idx / nc), a = (int)(idx - (long long)X * nc);
    double2* p = A + (size_t)X * 9 * nc * nc + (size_t)a * nc + a;
    p->x += dm;
}
void coarse_shift_mass(double2* A, int nc, double dm, const Geom& g, cudaStream_t st) {
    long long total = (long long)g.Vc * nc;
    note_launch();
    k_coarse_shift<<<(int)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(A, nc, dm, g.Vc);
}

// [X][d][a][b] <-> [X][d][b][a]
__global__ void k_transpose_blocks(double2* out, const double2* __restrict__ in, int nc, long long nblk) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= nblk * nc * nc) return;
    long long blk = idx / (nc * nc);
    int r = (int)(idx - blk * nc * nc);
    int i = r / nc, j = r - i * nc;
    out[blk * nc * nc + (size_t)j * nc + i] = in[idx];
}
void coarse_op_transpose(double2* out, const double2* in, int nc, int Vc, cudaStream_t st) {
    long long total = (long long)Vc * 9 * nc * nc;
    note_launch();
    k_transpose_blocks<<<(int)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(out, in, nc, (long long)Vc * 9);
}

// ================================================================ coarse apply
// y[X][a] = sum_d sum_b A[X][d][b][a] x[X+d][b]; one thread per (X, a), lanes
// read consecutive a (column-major blocks), x[X+d][b] is a warp broadcast.
// dag: sigma3 on x and on y.  FIN: 0 none, 1 ||y||^2 -> slot, 2 CG alpha,
// 3 CG beta (the CG variants are skipped once scal[S_CG_DONE] is set).
template <typename T, bool DAG, int FIN>
__global__ void __launch_bounds__(256) k_coarse_apply(v2<T>* __restrict__ y, const v2<T>* __restrict__ A,
                                                      const v2<T>* __restrict__ x, int nc, Geom g, int slot, Reduce R) {
    if (FIN >= 2 && R.scal[S_CG_DONE] != 0.0) return;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int nvh = nc >> 1;
    double red[1] = {0.0};
    if (idx < (long long)g.Vc * nc) {
        int X = (int)(idx / nc), a = (int)(idx - (long long)X * nc);
        cx<T> acc(0, 0);
        for (int d = 0; d < 9; ++d) {
            int Y = coarse_neighbour(g, X, d);
            const v2<T>* Ad = A + ((size_t)X * 9 + d) * nc * nc + a;
            const v2<T>* xY = x + (size_t)Y * nc;
            if (DAG) {
                for (int b = 0; b < nvh; ++b) cmad(acc, ldg<T>(Ad + (size_t)b * nc), ldg<T>(xY + b));
                for (int b = nvh; b < nc; ++b) {
                    cx<T> xb = ldg<T>(xY + b);
                    cmad(acc, ldg<T>(Ad + (size_t)b * nc), cx<T>(-xb.r, -xb.i));
                }
            } else {
                for (int b = 0; b < nc; ++b) cmad(acc, ldg<T>(Ad + (size_t)b * nc), ldg<T>(xY + b));
            }
        }
        if (DAG && a >= nvh) acc = cx<T>(-acc.r, -acc.i);
        st<T>(y + idx, acc);
        red[0] = (double)norm2(acc);
    }
    if (FIN == 1) {
        grid_reduce<1>(red, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) { R.scal[slot] = t[0]; });
    } else if (FIN == 2) {
        grid_reduce<1>(red, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) {
            if (t[0] > 0) R.scal[S_CG_ALPHA] = R.scal[S_CG_GAMMA] / t[0];
            else { R.scal[S_CG_ALPHA] = 0.0; R.scal[S_CG_DONE] = 1.0; }
        });
    } else if (FIN == 3) {
        grid_reduce<1>(red, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) {
            double gam = R.scal[S_CG_GAMMA];
            R.scal[S_CG_BETA] = gam > 0 ? t[0] / gam : 0.0;
            R.scal[S_CG_GAMMA] = t[0];
        });
    }
}

template <typename T>
void coarse_apply(v2<T>* y, const v2<T>* A, const v2<T>* x, int nc, bool dag, int slot, const Geom& g, const Reduce& R,
                  cudaStream_t st) {
    long long total = (long long)g.Vc * nc;
    int grid = (int)((total + kThreads - 1) / kThreads);
    if (slot >= 0) {
        if (dag) { note_launch(); k_coarse_apply<T, true, 1><<<grid, kThreads, 0, st>>>(y, A, x, nc, g, slot, R); }
        else { note_launch(); k_coarse_apply<T, false, 1><<<grid, kThreads, 0, st>>>(y, A, x, nc, g, slot, R); }
    } else {
        if (dag) { note_launch(); k_coarse_apply<T, true, 0><<<grid, kThreads, 0, st>>>(y, A, x, nc, g, slot, R); }
        else { note_launch(); k_coarse_apply<T, false, 0><<<grid, kThreads, 0, st>>>(y, A, x, nc, g, slot, R); }
    }
}

// ================================================================ CGNR (CGLS) on D_c
template <typename T>
__global__ void k_cg_start(v2<T>* __restrict__ y, v2<T>* __restrict__ r, const v2<T>* __restrict__ rc, size_t n,
                           double tol, int maxit, Reduce R) {
    T a = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        v2<T> v = rc[i];
        r[i] = v;
        v2<T> z; z.x = 0; z.y = 0;
        y[i] = z;
        a += v.x * v.x + v.y * v.y;
    }
    double acc[1] = {(double)a};
    grid_reduce<1>(acc, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) {
        R.scal[S_CG_RC2] = t[0];
        R.scal[S_CG_R2] = t[0];
        R.scal[S_CG_TOL2] = tol * tol;
        R.scal[S_CG_MAXIT] = (double)maxit;
        R.scal[S_CG_ITERS] = 0.0;
        R.scal[S_CG_DONE] = (t[0] > 0 && maxit > 0) ? 0.0 : 1.0;
    });
}
template <typename T>
__global__ void k_cg_copy(v2<T>* __restrict__ p, const v2<T>* __restrict__ s, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = s[i];
}
// y += alpha p; r -= alpha q; ||r||^2; iteration count and stopping test
template <typename T>
__global__ void k_cg_update1(v2<T>* __restrict__ y, v2<T>* __restrict__ r, const v2<T>* __restrict__ p,
                             const v2<T>* __restrict__ q, size_t n, Reduce R) {
    if (R.scal[S_CG_DONE] != 0.0) return;
    T al = (T)R.scal[S_CG_ALPHA];
    T a = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        st<T>(y + i, ld<T>(y + i) + al * ld<T>(p + i));
        cx<T> v = ld<T>(r + i) - al * ld<T>(q + i);
        st<T>(r + i, v);
        a += norm2(v);
    }
    double acc[1] = {(double)a};
    grid_reduce<1>(acc, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) {
        double it = R.scal[S_CG_ITERS] + 1.0;
        R.scal[S_CG_ITERS] = it;
        R.scal[S_CG_R2] = t[0];
        if (t[0] <= R.scal[S_CG_TOL2] * R.scal[S_CG_RC2] || it >= R.scal[S_CG_MAXIT]) R.scal[S_CG_DONE] = 1.0;
    });
}
// p = s + beta p
template <typename T>
__global__ void k_cg_update2(v2<T>* __restrict__ p, const v2<T>* __restrict__ s, size_t n, const double* __restrict__ scal) {
    if (scal[S_CG_DONE] != 0.0) return;
    T be = (T)scal[S_CG_BETA];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        st<T>(p + i, ld<T>(s + i) + be * ld<T>(p + i));
}

template <typename T>
void cg_init(v2<T>* y, v2<T>* r, const v2<T>* rc, size_t n, double tol, int maxit, const Reduce& R, cudaStream_t st) {
    note_launch();
    k_cg_start<T><<<reduce_grid(n), kThreads, 0, st>>>(y, r, rc, n, tol, maxit, R);
}
// s = D_c^dag r, gamma = ||s||^2, p = s
template <typename T>
void cg_first_direction(v2<T>* s, v2<T>* p, const v2<T>* r, const v2<T>* A, int nc, const Geom& g, const Reduce& R,
                        cudaStream_t st) {
    size_t n = (size_t)g.Vc * nc;
    coarse_apply<T>(s, A, r, nc, true, S_CG_GAMMA, g, R, st);
    note_launch();
    k_cg_copy<T><<<reduce_grid(n), kThreads, 0, st>>>(p, s, n);
}
template <typename T>
void cg_step(v2<T>* y, v2<T>* r, v2<T>* s, v2<T>* p, v2<T>* q, const v2<T>* A, int nc, const Geom& g, const Reduce& R,
             cudaStream_t st) {
    size_t n = (size_t)g.Vc * nc;
    int grid = (int)((n + kThreads - 1) / kThreads);
    note_launch();
    k_coarse_apply<T, false, 2><<<grid, kThreads, 0, st>>>(q, A, p, nc, g, -1, R);        // q = D_c p, alpha
    note_launch();
    k_cg_update1<T><<<reduce_grid(n), kThreads, 0, st>>>(y, r, p, q, n, R);               // y, r, stop test
    note_launch();
    k_coarse_apply<T, true, 3><<<grid, kThreads, 0, st>>>(s, A, r, nc, g, -1, R);         // s = D_c^dag r, beta
    note_launch();
    k_cg_update2<T><<<reduce_grid(n), kThreads, 0, st>>>(p, s, n, R.scal);                // p = s + beta p
}

#define INST(T)                                                                                                     \
    template void restrict_<T>(v2<T>*, const v2<T>*, const v2<T>*, int, const Geom&, cudaStream_t, int, int);       \
    template void prolong<T>(v2<T>*, const v2<T>*, const v2<T>*, int, const Geom&, cudaStream_t, int, int);         \
    template void coarse_apply<T>(v2<T>*, const v2<T>*, const v2<T>*, int, bool, int, const Geom&, const Reduce&,    \
                                  cudaStream_t);                                                                    \
    template void cg_init<T>(v2<T>*, v2<T>*, const v2<T>*, size_t, double, int, const Reduce&, cudaStream_t);       \
    template void cg_first_direction<T>(v2<T>*, v2<T>*, const v2<T>*, const v2<T>*, int, const Geom&, const Reduce&, \
                                        cudaStream_t);                                                              \
    template void cg_step<T>(v2<T>*, v2<T>*, v2<T>*, v2<T>*, v2<T>*, const v2<T>*, int, const Geom&, const Reduce&,  \
                             cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace wmg

namespace wmg {
// P64[X][s][i][k6][l] -> boundary [i][lex site][spin][colour] (zero on the other chirality)
__global__ void k_prolongator_to_boundary(double2* out, const double2* __restrict__ P, int nv, Geom g) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;   // over nv * V * 12 in internal order
    long long total = (long long)nv * g.V * 12;
    if (idx >= total) return;
    int i = (int)(idx / (g.V * 12));
    long long r = idx - (long long)i * g.V * 12;
    int X = (int)(r / (12LL * g.Vb));
    int rem = (int)(r - (long long)X * 12 * g.Vb);
    int k = rem / g.Vb, l = rem - k * g.Vb;
    int s = k / 6, kk = k - 6 * s;
    long long lex = lex_site(g, X, l);
    double2 v = P[((((size_t)X * 2 + s) * nv + i) * 6 + kk) * g.Vb + l];
    out[((size_t)i * g.V + lex) * 12 + 6 * s + kk] = v;
}
void prolongator_to_boundary(double2* out, const double2* P, int nv, const Geom& g, cudaStream_t st) {
    long long total = (long long)nv * g.V * 12;
    note_launch();
    k_prolongator_to_boundary<<<(int)((total + 255) / 256), 256, 0, st>>>(out, P, nv, g);
}
}  // namespace wmg

// ================================================================ persistent CGNR
// The whole coarse solve in one cooperative launch: G co-resident CTAs loop
// over the CGLS iterations, separated by grid barriers.  Every spin-wait is
// bounded: after kBarrierSpinLimit polls the CTA sets *err and returns, and
// CTAs waiting at a barrier return as soon as *err is set.  Reductions:
// each CTA writes its partial sum, and after the barrier every CTA adds all
// partials in the same order, so all CTAs take identical decisions.
namespace wmg {

// One CG phase on the aggregates of this CTA, `xpb` at a time: stage the
// operand on X and its 8 neighbours in shared memory, then apply the coarse
// stencil.  Thread (x, d, row group) accumulates R consecutive rows a of block
// A[X][d] (one 16-byte load carries rows a, a+1 of column b) with U
// independent loads in flight; shared memory sums the 9 directions.
// The operand is formed while staging (STAGE):
//   ST_P: pn = s + beta * p_old   (first iteration: pn = s); own entries -> p_new
//         output q = D_c pn;          partial sums: n0 = ||q||^2
//   ST_R: rn = r_old - alpha * q; own entries -> r_new, y += alpha * p_cur;
//         output s = D_c^dag rn;      partial sums: n0 = ||s||^2, n1 = ||rn||^2
//   ST_PLAIN: operand = in;          output out = D_c(^dag) in, n0 = ||out||^2
enum { ST_PLAIN = 0, ST_P = 1, ST_R = 2 };

template <typename T, bool H16 = false> struct RowsPerThread { static constexpr int value = H16 ? 4 : 2; };

template <typename T, int R> struct RowLoad;
template <> struct RowLoad<double, 2> {
    static __device__ __forceinline__ void load(const v2<double>* p, cx<double> (&v)[2]) {
        double2 a = __ldg(p), b = __ldg(p + 1);
        v[0] = cx<double>(a.x, a.y);
        v[1] = cx<double>(b.x, b.y);
    }
};
template <> struct RowLoad<float, 2> {
    static __device__ __forceinline__ void load(const v2<float>* p, cx<float> (&v)[2]) {
        float4 a = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = cx<float>(a.x, a.y);
        v[1] = cx<float>(a.z, a.w);
    }
};
// four consecutive rows of the FP16 operator in one 16-byte load
__device__ __forceinline__ void row_load16(const __half2* p, cx<float> (&v)[4]) {
    uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const __half2* h = reinterpret_cast<const __half2*>(&u);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float2 f = __half22float2(h[r]);
        v[r] = cx<float>(f.x, f.y);
    }
}

template <typename T> struct PhaseArgs {
    const v2<T>* in;       // ST_PLAIN operand
    const v2<T>* s;        // ST_P: s
    const v2<T>* p_old;    // ST_P: previous direction (ignored when first)
    v2<T>* p_new;          // ST_P: own entries of pn; ST_R: p_cur (read)
    const v2<T>* r_old;    // ST_R
    const v2<T>* q;        // ST_R
    v2<T>* r_new;          // ST_R
    v2<T>* y;              // ST_R
    v2<T>* out;            // result
    T coef;                // beta (ST_P) or alpha (ST_R)
    bool first;            // ST_P, first iteration
};

template <typename T, bool DAG, int STAGE, bool H16>
__device__ void cg_phase(const PhaseArgs<T>& ph, const v2<T>* __restrict__ A, const __half2* __restrict__ A16,
                         const float* __restrict__ s16, int nc, int xpb, const Geom& g, v2<T>* xs, cx<T>* part,
                         const int* __restrict__ nbr, T& n0, T& n1) {
    constexpr int R = RowsPerThread<T, H16>::value;
    const int nvh = nc >> 1, nrow = 9 * nc, ngrp = nc / R, nthr = 9 * ngrp, nall = xpb * nrow;
    const int xl = threadIdx.x / nthr, rem = threadIdx.x - xl * nthr;
    const int d = rem / ngrp, a0 = (rem - d * ngrp) * R;
    for (int Xb = blockIdx.x * xpb; Xb < g.Vc; Xb += gridDim.x * xpb) {
        for (int i = threadIdx.x; i < nall; i += blockDim.x) {
            int xi = i / nrow, ri = i - xi * nrow;
            int di = ri / nc, b = ri - di * nc;
            int X = Xb + xi;
            if (X < g.Vc) {
                int Y = __ldg(nbr + (size_t)X * 9 + di);
                size_t o = (size_t)Y * nc + b;
                cx<T> v;
                if (STAGE == ST_PLAIN) {
                    v = ld<T>(ph.in + o);
                } else if (STAGE == ST_P) {
                    v = ld<T>(ph.s + o);
                    if (!ph.first) v = v + ph.coef * ld<T>(ph.p_old + o);
                    if (di == 0) st<T>(ph.p_new + o, v);
                } else {
                    v = ld<T>(ph.r_old + o) - ph.coef * ld<T>(ph.q + o);
                    if (di == 0) {
                        st<T>(ph.r_new + o, v);
                        st<T>(ph.y + o, ld<T>(ph.y + o) + ph.coef * ld<T>(ph.p_new + o));
                        n1 += norm2(v);
                    }
                }
                if (DAG && b >= nvh) v = cx<T>(-v.r, -v.i);
                st<T>(xs + i, v);
            }
        }
        __syncthreads();
        const int X = Xb + xl;
        if (threadIdx.x < xpb * nthr && X < g.Vc) {
            const v2<T>* xd = xs + xl * nrow + d * nc;
            cx<T> acc[R][2];
#pragma unroll
            for (int r = 0; r < R; ++r) { acc[r][0] = cx<T>(0, 0); acc[r][1] = cx<T>(0, 0); }
            constexpr int U = 4;
            if constexpr (H16) {
                const __half2* Ad = A16 + ((size_t)X * 9 + d) * nc * nc + a0;
                for (int b0 = 0; b0 < nc; b0 += U) {
                    uint4 raw[U];
#pragma unroll
                    for (int j = 0; j < U; ++j)
                        if (b0 + j < nc) raw[j] = __ldg(reinterpret_cast<const uint4*>(Ad + (size_t)(b0 + j) * nc));
#pragma unroll
                    for (int j = 0; j < U; ++j)
                        if (b0 + j < nc) {
                            cx<T> xb = ld<T>(xd + b0 + j);
                            const __half2* h = reinterpret_cast<const __half2*>(&raw[j]);
#pragma unroll
                            for (int r = 0; r < R; ++r) {
                                float2 f = __half22float2(h[r]);
                                cmad(acc[r][j & 1], cx<T>(f.x, f.y), xb);
                            }
                        }
                }
                const T sc = (T)s16[(size_t)X * 9 + d];
#pragma unroll
                for (int r = 0; r < R; ++r) part[xl * nrow + d * nc + a0 + r] = sc * (acc[r][0] + acc[r][1]);
            } else {
                const v2<T>* Ad = A + ((size_t)X * 9 + d) * nc * nc + a0;
                for (int b0 = 0; b0 < nc; b0 += U) {
                    cx<T> av[U][R];
#pragma unroll
                    for (int j = 0; j < U; ++j)
                        if (b0 + j < nc) RowLoad<T, R>::load(Ad + (size_t)(b0 + j) * nc, av[j]);
#pragma unroll
                    for (int j = 0; j < U; ++j)
                        if (b0 + j < nc) {
                            cx<T> xb = ld<T>(xd + b0 + j);
#pragma unroll
                            for (int r = 0; r < R; ++r) cmad(acc[r][j & 1], av[j][r], xb);
                        }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) part[xl * nrow + d * nc + a0 + r] = acc[r][0] + acc[r][1];
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < xpb * nc; t += blockDim.x) {
            int x2 = t / nc, a2 = t - x2 * nc;
            int X2 = Xb + x2;
            if (X2 < g.Vc) {
                cx<T> sum = part[x2 * nrow + a2];
#pragma unroll
                for (int dd = 1; dd < 9; ++dd) sum = sum + part[x2 * nrow + dd * nc + a2];
                if (DAG && a2 >= nvh) sum = cx<T>(-sum.r, -sum.i);
                st<T>(ph.out + (size_t)X2 * nc + a2, sum);
                n0 += norm2(sum);
            }
        }
        __syncthreads();
    }
}

// CGLS (CG on the normal equations), the textbook recurrences
//   q = D_c p, alpha = gamma/||q||^2, y += alpha p, r -= alpha q,
//   s = D_c^dag r, beta = ||s||^2/gamma, p = s + beta p
// with two grid barriers per iteration: the elementwise updates of p and r are
// done while staging the neighbour operands of the next stencil (p and r
// double-buffered so that no CTA overwrites what another still reads).
template <typename T> struct CgnrMaxThreads { static constexpr int value = 384; };

template <typename T, bool H16>
__global__ void __launch_bounds__(CgnrMaxThreads<T>::value, 2) k_cgnr_persistent(CgnrArgs<T> a) {
    extern __shared__ unsigned char smem_raw[];
    const int nc = a.nc, xpb = a.xpb;
    v2<T>* xs = reinterpret_cast<v2<T>*>(smem_raw);
    cx<T>* part = reinterpret_cast<cx<T>*>(smem_raw + sizeof(v2<T>) * 9 * nc * xpb);
    __shared__ T shr[33];
    const unsigned int G = gridDim.x;
    unsigned int* cnt = a.bar;
    unsigned int* gen = a.bar + 1;
    v2<T>* rbuf[2] = {a.r, a.r1};
    v2<T>* pbuf[2] = {a.p, a.p1};
    // y = 0, r = rc on the aggregates of this CTA; ||rc||^2
    T loc = 0;
    for (int Xb = blockIdx.x * xpb; Xb < a.g.Vc; Xb += G * xpb)
        for (int t = threadIdx.x; t < xpb * nc; t += blockDim.x) {
            int X = Xb + t / nc;
            if (X < a.g.Vc) {
                size_t o = (size_t)X * nc + (t % nc);
                v2<T> v = a.rc[o];
                a.r[o] = v;
                v2<T> z; z.x = 0; z.y = 0;
                a.y[o] = z;
                loc += v.x * v.x + v.y * v.y;
            }
        }
    write_partial<T>(loc, a.partials, 0, shr);
    if (!grid_sync(cnt, gen, G, a.err)) return;
    const T rc2 = sum_partials<T>(a.partials, 0, G, shr);
    int it = 0;
    T r2 = rc2;
    if (rc2 > T(0) && a.maxit > 0) {
        PhaseArgs<T> ph{};
        T n0 = 0, n1 = 0;
        // s = D_c^dag r, gamma = ||s||^2
        ph.in = a.r;
        ph.out = a.s;
        cg_phase<T, true, ST_PLAIN, H16>(ph, a.A, a.A16, a.s16, nc, xpb, a.g, xs, part, a.nbr, n0, n1);
        write_partial<T>(n0, a.partials, 1, shr);
        if (!grid_sync(cnt, gen, G, a.err)) return;
        T gamma = sum_partials<T>(a.partials, 1, G, shr);
        T beta = 0;
        for (;;) {
            const int b = it & 1;
            // p = s + beta p; q = D_c p
            ph = PhaseArgs<T>{};
            ph.s = a.s; ph.p_old = pbuf[b ^ 1]; ph.p_new = pbuf[b]; ph.out = a.q;
            ph.coef = beta; ph.first = (it == 0);
            n0 = 0; n1 = 0;
            cg_phase<T, false, ST_P, H16>(ph, a.A, a.A16, a.s16, nc, xpb, a.g, xs, part, a.nbr, n0, n1);
            write_partial<T>(n0, a.partials, 0, shr);
            if (!grid_sync(cnt, gen, G, a.err)) return;
            T qq = sum_partials<T>(a.partials, 0, G, shr);
            if (!(qq > T(0))) break;
            T alpha = gamma / qq;
            // y += alpha p; r -= alpha q; s = D_c^dag r
            ph = PhaseArgs<T>{};
            ph.r_old = rbuf[b]; ph.q = a.q; ph.r_new = rbuf[b ^ 1]; ph.y = a.y; ph.p_new = pbuf[b];
            ph.out = a.s; ph.coef = alpha;
            n0 = 0; n1 = 0;
            cg_phase<T, true, ST_R, H16>(ph, a.A, a.A16, a.s16, nc, xpb, a.g, xs, part, a.nbr, n0, n1);
            write_partial<T>(n0, a.partials, 1, shr);
            write_partial<T>(n1, a.partials, 2, shr);
            if (!grid_sync(cnt, gen, G, a.err)) return;
            T gnew = sum_partials<T>(a.partials, 1, G, shr);
            r2 = sum_partials<T>(a.partials, 2, G, shr);
            ++it;
            if (r2 <= (T)a.tol2 * rc2 || it >= a.maxit) break;
            beta = gnew / gamma;
            gamma = gnew;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.scal[S_CG_ITERS] = (double)it;
        a.scal[S_CG_R2] = (double)r2;
        a.scal[S_CG_RC2] = (double)rc2;
        a.scal[S_CG_DONE] = 1.0;
        a.scal[S_CG_TOTAL] += (double)it;
    }
}

// aggregates per CTA: as many 9*nc-thread groups as fit in the thread limit
template <typename T, bool H16> int cgnr_threads_per_x(int nc) { return 9 * (nc / RowsPerThread<T, H16>::value); }
template <typename T, bool H16> int cgnr_xpb(int nc) {
    int x = CgnrMaxThreads<T>::value / cgnr_threads_per_x<T, H16>(nc);
    return x > 0 ? x : 1;
}
template <typename T, bool H16> int cgnr_block_threads(int nc) {
    return ((cgnr_xpb<T, H16>(nc) * cgnr_threads_per_x<T, H16>(nc) + 31) / 32) * 32;
}
template <typename T, bool H16> size_t cgnr_smem(int nc) {
    return (sizeof(v2<T>) + sizeof(cx<T>)) * 9 * (size_t)nc * cgnr_xpb<T, H16>(nc);
}

// co-resident CTAs for this nc, then the smallest balanced grid covering all aggregates
template <typename T, bool H16> int cgnr_grid(int nc, int Vc) {
    // per device (SM count and occupancy may differ between devices); slots are
    // atomic so host threads calling at once see either 0 or the final value
    constexpr int kDevs = 16;
    static std::atomic<int> cached[kDevs][2][128];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) return 0;
    int key = nc < 128 ? nc : 127;
    std::atomic<int>& slot = cached[dev][H16 ? 1 : 0][key];
    int gmax = slot.load(std::memory_order_acquire);
    if (gmax == 0) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        size_t sm = cgnr_smem<T, H16>(nc);   // < 48 KB: no attribute needed
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cgnr_persistent<T, H16>, cgnr_block_threads<T, H16>(nc), sm);
        gmax = per * sms;
        slot.store(gmax, std::memory_order_release);
    }
    if (gmax <= 0) return 0;
    int xpb = cgnr_xpb<T, H16>(nc);
    int batches = (Vc + xpb - 1) / xpb;               // CTA-sized pieces of work
    int rounds = (batches + gmax - 1) / gmax;         // pieces per CTA
    return (batches + rounds - 1) / rounds;
}

template <typename T, bool H16> cudaError_t cgnr_launch(const CgnrArgs<T>& args, cudaStream_t st) {
    int G = cgnr_grid<T, H16>(args.nc, args.g.Vc);
    if (G <= 0) return cudaErrorCooperativeLaunchTooLarge;
    CgnrArgs<T> a = args;
    a.xpb = cgnr_xpb<T, H16>(a.nc);
    void* params[] = {&a};
    note_launch();
    return cudaLaunchCooperativeKernel((const void*)k_cgnr_persistent<T, H16>, dim3(G),
                                       dim3(cgnr_block_threads<T, H16>(a.nc)), params, cgnr_smem<T, H16>(a.nc), st);
}
template <> cudaError_t cgnr_persistent<float>(const CgnrArgs<float>& a, cudaStream_t st) {
    if (a.A16) {
        if (a.nc % 4 != 0) return cudaErrorInvalidValue;
        return cgnr_launch<float, true>(a, st);
    }
    return cgnr_launch<float, false>(a, st);
}
template <> cudaError_t cgnr_persistent<double>(const CgnrArgs<double>& a, cudaStream_t st) {
    return cgnr_launch<double, false>(a, st);
}

// coarse neighbour table nbr[X][d] (d = 0 self, 1+2mu / 2+2mu: +mu / -mu)
__global__ void k_coarse_nbr(int* nbr, Geom g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.Vc * 9) nbr[i] = coarse_neighbour(g, i / 9, i % 9);
}
void coarse_neighbour_table(int* nbr, const Geom& g, cudaStream_t st) {
    note_launch();
    k_coarse_nbr<<<(g.Vc * 9 + 255) / 256, 256, 0, st>>>(nbr, g);
}

// FP16 copy of the coarse operator with one scale per (X, d) block: A16 = A / s, s = max |Re, Im|
__global__ void k_coarse_pack16(__half2* A16, float* s16, const double2* __restrict__ A, int nc) {
    __shared__ double sh[33];
    const size_t blk = blockIdx.x, nn = (size_t)nc * nc;
    const double2* Ab = A + blk * nn;
    double mx = 0;
    for (size_t i = threadIdx.x; i < nn; i += blockDim.x) mx = fmax(mx, fmax(fabs(Ab[i].x), fabs(Ab[i].y)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
        sh[32] = m > 0 ? m : 1.0;
        s16[blk] = (float)sh[32];
    }
    __syncthreads();
    const double inv = 1.0 / (double)(float)sh[32];
    for (size_t i = threadIdx.x; i < nn; i += blockDim.x)
        A16[blk * nn + i] = __floats2half2_rn((float)(Ab[i].x * inv), (float)(Ab[i].y * inv));
}
void coarse_pack16(__half2* A16, float* s16, const double2* A, int nc, int Vc, cudaStream_t st) {
    note_launch();
    k_coarse_pack16<<<Vc * 9, 256, 0, st>>>(A16, s16, A, nc);
}



}  // namespace wmg

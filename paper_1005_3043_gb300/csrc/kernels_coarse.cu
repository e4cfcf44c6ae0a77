// Transfer and coarse-level kernels: block orthonormalisation of the
// prototypes (eq. 4 with the chirality split), restriction r_c = P^dag r,
// prolongation e = P y, the Galerkin coarse operator D_c = P^dag D P and its
// nearest-neighbour application, and the CGNR (CGLS) coarse solve steps.
#include "mg_launch.h"

namespace wmg {

constexpr int kThreads = 256;

static inline int reduce_grid(size_t n) {
    size_t b = (n + kThreads - 1) / kThreads;
    if (b > (size_t)kMaxReduceBlocks) b = kMaxReduceBlocks;
    return (int)(b > 0 ? b : 1);
}

// ================================================================ block orthonormalisation
// One CTA per (aggregate X, chirality s).  Column i of the panel is prototype i
// restricted to X and to the spins of s (6*Vb complex).  Modified Gram-Schmidt
// applied twice in index order, then normalisation: the Q factor with a
// positive real R-diagonal.  Each thread keeps its elements of the current
// column in registers; earlier columns are re-read from the output.
constexpr int kOrthoMaxPerThread = 8;

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
__device__ __forceinline__ cx<double> block_sum2(cx<double> v, double* sh) {
    double a[2] = {v.r, v.i};
    block_reduce<2>(a, (double (*)[32])sh);
    __syncthreads();
    if (threadIdx.x == 0) { sh[64] = a[0]; sh[65] = a[1]; }
    __syncthreads();
    cx<double> r(sh[64], sh[65]);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) k_block_ortho(double2* __restrict__ P, const double2* __restrict__ Vin, int nv,
                                                     Geom g, int* status) {
    __shared__ double sh[2 * 32 + 2];
    int X = blockIdx.x >> 1, s = blockIdx.x & 1;
    int len = 6 * g.Vb;
    size_t vstride = (size_t)g.Vc * 12 * g.Vb;       // one prototype
    double2* panel = P + ((size_t)X * 2 + s) * nv * len;
    cx<double> w[kOrthoMaxPerThread];
    for (int i = 0; i < nv; ++i) {
        const double2* vi = Vin + (size_t)i * vstride + ((size_t)X * 12 + 6 * s) * g.Vb;   // k = 6s..6s+5 contiguous
        double n0 = 0;
#pragma unroll
        for (int q = 0; q < kOrthoMaxPerThread; ++q) {
            int e = threadIdx.x + q * blockDim.x;
            w[q] = e < len ? ld<double>(vi + e) : cx<double>(0, 0);
            n0 += norm2(w[q]);
        }
        n0 = block_sum(n0, sh);
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < i; ++j) {
                const double2* qj = panel + (size_t)j * len;
                cx<double> c(0, 0);
#pragma unroll
                for (int q = 0; q < kOrthoMaxPerThread; ++q) {
                    int e = threadIdx.x + q * blockDim.x;
                    if (e < len) cmadc(c, ld<double>(qj + e), w[q]);
                }
                c = block_sum2(c, sh);
#pragma unroll
                for (int q = 0; q < kOrthoMaxPerThread; ++q) {
                    int e = threadIdx.x + q * blockDim.x;
                    if (e < len) w[q] = w[q] - c * ld<double>(qj + e);
                }
            }
        double n = 0;
#pragma unroll
        for (int q = 0; q < kOrthoMaxPerThread; ++q) n += norm2(w[q]);
        n = sqrt(block_sum(n, sh));
        if (!(n > 1e-12 * sqrt(n0))) {
            if (threadIdx.x == 0) atomicExch(status, 1);
            n = 1.0;
        }
        double f = 1.0 / n;
        double2* qi = panel + (size_t)i * len;
#pragma unroll
        for (int q = 0; q < kOrthoMaxPerThread; ++q) {
            int e = threadIdx.x + q * blockDim.x;
            if (e < len) st<double>(qi + e, f * w[q]);
        }
        __syncthreads();   // column i visible to the block before it is re-read
    }
}

void block_orthonormalize(double2* P, const double2* V, int nv, const Geom& g, int* d_status, cudaStream_t st) {
    k_block_ortho<<<2 * g.Vc, kThreads, 0, st>>>(P, V, nv, g, d_status);
}

// ================================================================ restriction / prolongation
// r_c[X][s*Nv + i] = <P_(X,s,i), r>: one CTA per (X, s); the chirality-s half of
// r on X (6*Vb contiguous) is staged in shared memory, warp w handles i = w, w+8, ...
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(v2<T>* __restrict__ rc, const v2<T>* __restrict__ P,
                                                  const v2<T>* __restrict__ r, int nv, Geom g) {
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
            rc[(size_t)X * 2 * nv + s * nv + i] = o;
        }
    }
}
// e[X][k][l] = sum_i P[X][s(k)][i][k%6][l] y[X][s(k)*Nv + i]
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(v2<T>* __restrict__ e, const v2<T>* __restrict__ P,
                                                 const v2<T>* __restrict__ yc, int nv, Geom g) {
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
    const v2<T>* y = yc + (size_t)X * 2 * nv + s * nv;
    cx<T> a(0, 0);
    for (int i = 0; i < nv; ++i) cmad(a, ldg<T>(p + (size_t)i * len), ldg<T>(y + i));
    st<T>(e + idx, a);
}

template <typename T> void restrict_(v2<T>* rc, const v2<T>* P, const v2<T>* r, int nv, const Geom& g, cudaStream_t st) {
    size_t sm = sizeof(v2<T>) * 6 * g.Vb;
    k_restrict<T><<<2 * g.Vc, kThreads, sm, st>>>(rc, P, r, nv, g);
}
template <typename T> void prolong(v2<T>* e, const v2<T>* P, const v2<T>* yc, int nv, const Geom& g, cudaStream_t st) {
    long long total = g.V * 12;
    k_prolong<T><<<(int)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(e, P, yc, nv, g);
}

// ================================================================ coarse operator build
// One CTA per (aggregate X, hop h = 2*mu + (0 fwd | 1 bwd)).  For site chunks
// of X it forms W_b(x) = H_h(x) P_b(y) for every coarse column b (H_h the
// hop of eq. 2 from x to y = x +/- mu, P_b column b at y) and accumulates
// conj(P_a(x)) . W_b(x) over the 6 components of chirality s_a.  Hops leaving
// X through its face in direction h go to A[X][1+h]; hops staying inside X go
// to Aself[X][h] (summed later with the diagonal (4+m)).  FP64 throughout.
constexpr int kBuildChunk = 8;

template <int MU, bool FWD>
__device__ __forceinline__ void hop_column(const cx<double> (&p)[4][3], const double2* __restrict__ u, int Vb,
                                           double coef, cx<double> (&out)[4][3]) {
    // spin projection (same convention as the fine operator)
    cx<double> h[2][3];
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
    cx<double> w[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w[0][a] = cx<double>(0, 0);
        w[1][a] = cx<double>(0, 0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (FWD) {
                cx<double> uab = ld<double>(u + (3 * a + b) * Vb);
                cmad(w[0][a], uab, h[0][b]);
                cmad(w[1][a], uab, h[1][b]);
            } else {
                cx<double> uba = ld<double>(u + (3 * b + a) * Vb);
                cmadc(w[0][a], uba, h[0][b]);
                cmadc(w[1][a], uba, h[1][b]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<double> w0 = coef * w[0][c], w1 = coef * w[1][c];
        out[0][c] = w0;
        out[1][c] = w1;
        if (MU == 0) { out[2][c] = FWD ? mul_i(w1) : mul_mi(w1); out[3][c] = FWD ? mul_i(w0) : mul_mi(w0); }
        else if (MU == 1) { out[2][c] = FWD ? cx<double>(-w1.r, -w1.i) : w1; out[3][c] = FWD ? w0 : cx<double>(-w0.r, -w0.i); }
        else if (MU == 2) { out[2][c] = FWD ? mul_i(w0) : mul_mi(w0); out[3][c] = FWD ? mul_mi(w1) : mul_i(w1); }
        else { out[2][c] = FWD ? cx<double>(-w0.r, -w0.i) : w0; out[3][c] = FWD ? cx<double>(-w1.r, -w1.i) : w1; }
    }
}

template <int MU, bool FWD>
__device__ void build_hop(double2* __restrict__ A, double2* __restrict__ Aself, const double2* __restrict__ P,
                          const double2* __restrict__ U, int nv, const Geom& g, int X, int h, double2* Wsh,
                          double2* Psh, unsigned char* leaves) {
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
        // W_b(x) for x in chunk, all columns b: Wsh[(xi*nc + b)*12 + k]
        for (int t = threadIdx.x; t < cs * nc; t += blockDim.x) {
            int xi = t / nc, b = t - xi * nc;
            int l = l0 + xi;
            int lc[4];
            local_coords(g, l, lc);
            int Xn, ln;
            bool flip;
            neighbour(g, X, l, lc, xcX, MU, FWD ? 1 : -1, Xn, ln, flip);
            if (b == 0) leaves[xi] = (Xn != X || (FWD ? lc[MU] == g.B[MU] - 1 : lc[MU] == 0)) ? 1 : 0;
            int sb = b / nv, ib = b - sb * nv;
            cx<double> p[4][3];
            const double2* col = P + (((size_t)Xn * 2 + sb) * nv + ib) * len;
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    int s_sp = sp >> 1;
                    p[sp][c] = (s_sp == sb) ? ld<double>(col + ((sp & 1) * 3 + c) * g.Vb + ln) : cx<double>(0, 0);
                }
            const double2* u = FWD ? U + ((size_t)MU * g.Vc + X) * 9 * g.Vb + l : U + ((size_t)MU * g.Vc + Xn) * 9 * g.Vb + ln;
            cx<double> o[4][3];
            hop_column<MU, FWD>(p, u, g.Vb, flip ? 0.5 : -0.5, o);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) st<double>(Wsh + ((size_t)xi * nc + b) * 12 + 3 * sp + c, o[sp][c]);
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
                for (int xi = 0; xi < cs; ++xi) {
                    cx<double> t(0, 0);
#pragma unroll
                    for (int kk = 0; kk < 6; ++kk)
                        cmadc(t, ld<double>(Psh + ((size_t)xi * nc + a) * 6 + kk),
                              ld<double>(Wsh + ((size_t)xi * nc + b) * 12 + 6 * sa + kk));
                    if (leaves[xi]) acc_out[q] = acc_out[q] + t;
                    else acc_in[q] = acc_in[q] + t;
                }
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

__global__ void __launch_bounds__(256) k_coarse_hop(double2* A, double2* Aself, const double2* __restrict__ P,
                                                    const double2* __restrict__ U, int nv, Geom g) {
    extern __shared__ unsigned char smem_raw[];
    const int nc = 2 * nv;
    double2* Wsh = reinterpret_cast<double2*>(smem_raw);
    double2* Psh = Wsh + (size_t)kBuildChunk * nc * 12;
    unsigned char* leaves = reinterpret_cast<unsigned char*>(Psh + (size_t)kBuildChunk * nc * 6);
    int X = blockIdx.x >> 3, h = blockIdx.x & 7;
    switch (h) {
        case 0: build_hop<0, true>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 1: build_hop<0, false>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 2: build_hop<1, true>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 3: build_hop<1, false>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 4: build_hop<2, true>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 5: build_hop<2, false>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        case 6: build_hop<3, true>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
        default: build_hop<3, false>(A, Aself, P, U, nv, g, X, h, Wsh, Psh, leaves); break;
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

void coarse_build(double2* A, double2* Aself, const double2* P, const double2* U, int nv, double mass, const Geom& g,
                  cudaStream_t st) {
    int nc = 2 * nv;
    size_t sm = sizeof(double2) * kBuildChunk * nc * 18 + kBuildChunk + 16;
    cudaFuncSetAttribute(k_coarse_hop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_coarse_hop<<<g.Vc * 8, kThreads, sm, st>>>(A, Aself, P, U, nv, g);
    long long total = (long long)g.Vc * nc * nc;
    k_coarse_diag<<<(int)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(A, Aself, nc, 4.0 + mass, g);
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
        grid_reduce<1>(red, R.partials, R.ticket, [&](double (&t)[1]) { R.scal[slot] = t[0]; });
    } else if (FIN == 2) {
        grid_reduce<1>(red, R.partials, R.ticket, [&](double (&t)[1]) {
            if (t[0] > 0) R.scal[S_CG_ALPHA] = R.scal[S_CG_GAMMA] / t[0];
            else { R.scal[S_CG_ALPHA] = 0.0; R.scal[S_CG_DONE] = 1.0; }
        });
    } else if (FIN == 3) {
        grid_reduce<1>(red, R.partials, R.ticket, [&](double (&t)[1]) {
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
        if (dag) k_coarse_apply<T, true, 1><<<grid, kThreads, 0, st>>>(y, A, x, nc, g, slot, R);
        else k_coarse_apply<T, false, 1><<<grid, kThreads, 0, st>>>(y, A, x, nc, g, slot, R);
    } else {
        if (dag) k_coarse_apply<T, true, 0><<<grid, kThreads, 0, st>>>(y, A, x, nc, g, slot, R);
        else k_coarse_apply<T, false, 0><<<grid, kThreads, 0, st>>>(y, A, x, nc, g, slot, R);
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
    grid_reduce<1>(acc, R.partials, R.ticket, [&](double (&t)[1]) {
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
    grid_reduce<1>(acc, R.partials, R.ticket, [&](double (&t)[1]) {
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
    k_cg_start<T><<<reduce_grid(n), kThreads, 0, st>>>(y, r, rc, n, tol, maxit, R);
}
// s = D_c^dag r, gamma = ||s||^2, p = s
template <typename T>
void cg_first_direction(v2<T>* s, v2<T>* p, const v2<T>* r, const v2<T>* A, int nc, const Geom& g, const Reduce& R,
                        cudaStream_t st) {
    size_t n = (size_t)g.Vc * nc;
    coarse_apply<T>(s, A, r, nc, true, S_CG_GAMMA, g, R, st);
    k_cg_copy<T><<<reduce_grid(n), kThreads, 0, st>>>(p, s, n);
}
template <typename T>
void cg_step(v2<T>* y, v2<T>* r, v2<T>* s, v2<T>* p, v2<T>* q, const v2<T>* A, int nc, const Geom& g, const Reduce& R,
             cudaStream_t st) {
    size_t n = (size_t)g.Vc * nc;
    int grid = (int)((n + kThreads - 1) / kThreads);
    k_coarse_apply<T, false, 2><<<grid, kThreads, 0, st>>>(q, A, p, nc, g, -1, R);        // q = D_c p, alpha
    k_cg_update1<T><<<reduce_grid(n), kThreads, 0, st>>>(y, r, p, q, n, R);               // y, r, stop test
    k_coarse_apply<T, true, 3><<<grid, kThreads, 0, st>>>(s, A, r, nc, g, -1, R);         // s = D_c^dag r, beta
    k_cg_update2<T><<<reduce_grid(n), kThreads, 0, st>>>(p, s, n, R.scal);                // p = s + beta p
}

#define INST(T)                                                                                                     \
    template void restrict_<T>(v2<T>*, const v2<T>*, const v2<T>*, int, const Geom&, cudaStream_t);                 \
    template void prolong<T>(v2<T>*, const v2<T>*, const v2<T>*, int, const Geom&, cudaStream_t);                   \
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
    k_prolongator_to_boundary<<<(int)((total + 255) / 256), 256, 0, st>>>(out, P, nv, g);
}
}  // namespace wmg

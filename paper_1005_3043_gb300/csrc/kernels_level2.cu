// Level 2 of the three-level method (Sec. III: the coarsening recursed with
// the chiral components kept separate; Sec. IV: 3-level W-cycle).
//
// Level-1 vectors are the coarse vectors of the two-level method, y[X1][2 Nv1]
// with X1 lexicographic over the level-1 lattice and dof a of chirality
// a / Nv1.  The level-1 lattice is cut into aggregates of block2 sites; the
// geometry g2 describes that blocking (L = level-1 extents, B = block2,
// Lc = level-2 extents, Vb = sites per level-2 aggregate, Vc = level-2 sites,
// V = level-1 sites).
//   P2[X2][s][i][k]  k = l2 * Nv1 + j: column (X2, s, i) of the level-2
//                    prolongator on the level-1 site l2 of aggregate X2 and
//                    dof s Nv1 + j (one contiguous panel per (X2, s))
//   A2[X2][d][b][a]  column-major 2Nv2 x 2Nv2 blocks, as D_c
#include "mg_launch.h"

namespace wmg {

constexpr int kL2Threads = 256;
constexpr int kL2MaxEntries = 16;   // A2 entries per thread in the build: (2 Nv2)^2 <= 16 * 256

__device__ __forceinline__ void level1_to_level2(const Geom& g2, int X1, int& X2, int& l2) {
    int c[4];
    int r = X1;
    for (int m = 0; m < 4; ++m) { c[m] = r % g2.L[m]; r /= g2.L[m]; }
    X2 = 0;
    l2 = 0;
    for (int m = 3; m >= 0; --m) {
        X2 = X2 * g2.Lc[m] + c[m] / g2.B[m];
        l2 = l2 * g2.B[m] + c[m] % g2.B[m];
    }
}

// complex sum over the CTA, returned to every thread
__device__ __forceinline__ cx<double> cta_sum2(cx<double> v, double* sh) {
    double a[2] = {v.r, v.i};
    block_reduce<2>(a, (double (*)[32])sh);
    __syncthreads();
    if (threadIdx.x == 0) { sh[64] = a[0]; sh[65] = a[1]; }
    __syncthreads();
    cx<double> r(sh[64], sh[65]);
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- block orthonormalisation (eq. 4 one level down)
// One CTA per (X2, s): the Nv2 columns are gathered into their panel of P2,
// then modified Gram-Schmidt twice in index order and normalisation (positive
// real R diagonal), in place, FP64.  *status = 1 when a column's norm falls
// below 1e-12 of its gathered norm.
__global__ void __launch_bounds__(kL2Threads) k_block_ortho_l2(double2* __restrict__ P2, const double2* __restrict__ V2,
                                                               int nv1, int nv2, Geom g2, int* status) {
    __shared__ double sh[2 * 32 + 2];
    const int X2 = blockIdx.x >> 1, s = blockIdx.x & 1, nc1 = 2 * nv1;
    const int len = g2.Vb * nv1;
    double2* panel = P2 + ((size_t)X2 * 2 + s) * nv2 * len;
    for (int i = 0; i < nv2; ++i)
        for (int k = threadIdx.x; k < len; k += blockDim.x) {
            const int l2 = k / nv1, j = k - l2 * nv1;
            const long long X1 = lex_site(g2, X2, l2);
            panel[(size_t)i * len + k] = V2[((size_t)i * g2.V + X1) * nc1 + s * nv1 + j];
        }
    __syncthreads();
    // Gram-Schmidt twice in index order, all projections of a pass at once
    // (classical form; the unique Q with positive real R-diagonal, as modified
    // Gram-Schmidt twice up to rounding): warp w forms c_j for j = w, w + nw, ...
    __shared__ double2 cj[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = 0; i < nv2; ++i) {
        double2* wi = panel + (size_t)i * len;
        double n0 = 0;
        for (int k = threadIdx.x; k < len; k += blockDim.x) n0 += wi[k].x * wi[k].x + wi[k].y * wi[k].y;
        const double orig = sqrt(cta_sum2(cx<double>(n0, 0), sh).r);
        for (int pass = 0; pass < 2 && i > 0; ++pass) {
            for (int j = warp; j < i; j += nw) {
                const double2* qj = panel + (size_t)j * len;
                cx<double> c(0, 0);
                for (int k = lane; k < len; k += 32) cmadc(c, ld<double>(qj + k), ld<double>(wi + k));
                c.r = warp_sum(c.r);
                c.i = warp_sum(c.i);
                if (lane == 0) cj[j] = make_double2(c.r, c.i);
            }
            __syncthreads();
            for (int k = threadIdx.x; k < len; k += blockDim.x) {
                cx<double> w = ld<double>(wi + k);
                for (int j = 0; j < i; ++j) w = w - cx<double>(cj[j].x, cj[j].y) * ld<double>(panel + (size_t)j * len + k);
                st<double>(wi + k, w);
            }
            __syncthreads();
        }
        double n1 = 0;
        for (int k = threadIdx.x; k < len; k += blockDim.x) n1 += wi[k].x * wi[k].x + wi[k].y * wi[k].y;
        double nrm = sqrt(cta_sum2(cx<double>(n1, 0), sh).r);
        if (!(nrm > 1e-12 * orig)) {
            if (threadIdx.x == 0) atomicExch(status, 1);
            nrm = 1.0;
        }
        const double inv = 1.0 / nrm;
        for (int k = threadIdx.x; k < len; k += blockDim.x) st<double>(wi + k, inv * ld<double>(wi + k));
        __syncthreads();
    }
}

// ---------------------------------------------------------------- transfers
// r2[X2][s Nv2 + i] = sum_k conj(P2[X2][s][i][k]) r1[X1(X2, l2)][s Nv1 + j]: one
// CTA per X2, one warp per output entry at a time
template <typename T>
__global__ void __launch_bounds__(kL2Threads) k_restrict_l2(v2<T>* __restrict__ r2, const v2<T>* __restrict__ P2,
                                                            const v2<T>* __restrict__ r1, int nv1, int nv2, Geom g2) {
    const int X2 = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nc1 = 2 * nv1, nc2 = 2 * nv2, len = g2.Vb * nv1;
    for (int o = warp; o < nc2; o += nw) {
        const int s = o / nv2, i = o - s * nv2;
        const v2<T>* col = P2 + (((size_t)X2 * 2 + s) * nv2 + i) * len;
        cx<T> acc(0, 0);
        for (int k = lane; k < len; k += 32) {
            const int l2 = k / nv1, j = k - l2 * nv1;
            const long long X1 = lex_site(g2, X2, l2);
            cmadc(acc, ldg<T>(col + k), ldg<T>(r1 + (size_t)X1 * nc1 + s * nv1 + j));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            acc.r += __shfl_xor_sync(0xffffffffu, acc.r, off);
            acc.i += __shfl_xor_sync(0xffffffffu, acc.i, off);
        }
        if (lane == 0) st<T>(r2 + (size_t)X2 * nc2 + o, acc);
    }
}
// e1[X1][a] = sum_i P2[X2][s][i][l2 Nv1 + j] y2[X2][s Nv2 + i], a = s Nv1 + j
template <typename T>
__global__ void __launch_bounds__(kL2Threads) k_prolong_l2(v2<T>* __restrict__ e1, const v2<T>* __restrict__ P2,
                                                           const v2<T>* __restrict__ y2, int nv1, int nv2, Geom g2) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nc1 = 2 * nv1, nc2 = 2 * nv2, len = g2.Vb * nv1;
    if (idx >= g2.V * nc1) return;
    const int X1 = (int)(idx / nc1), a = (int)(idx - (long long)X1 * nc1);
    const int s = a / nv1, j = a - s * nv1;
    int X2, l2;
    level1_to_level2(g2, X1, X2, l2);
    const v2<T>* col = P2 + ((size_t)X2 * 2 + s) * nv2 * len + (size_t)l2 * nv1 + j;
    const v2<T>* y = y2 + (size_t)X2 * nc2 + s * nv2;
    cx<T> acc(0, 0);
    for (int i = 0; i < nv2; ++i) cmad(acc, ldg<T>(col + (size_t)i * len), ldg<T>(y + i));
    st<T>(e1 + idx, acc);
}

// ---------------------------------------------------------------- Galerkin operator A2 = P2^dag A1 P2
// One CTA per (X2, d).  For every level-1 site x of X2 and stencil term t of A1
// whose slot is d (t = 0 and the terms that stay inside X2 land in d = 0, a
// term leaving X2 through the face of direction t in d = t), the products
// HP = A1[x][t] P2(x + t) (2Nv1 x 2Nv2) and the rows of P2 at x are staged in
// shared memory and every thread adds conj(P2_a(x)) HP_b to its entries (a, b).
// FP64 throughout.
__global__ void __launch_bounds__(kL2Threads) k_build_l2(double2* __restrict__ A2, const double2* __restrict__ P2,
                                                         const double2* __restrict__ A1, int nv1, int nv2, Geom g1,
                                                         Geom g2) {
    extern __shared__ __align__(16) unsigned char smem_l2[];
    const int nc1 = 2 * nv1, nc2 = 2 * nv2, len = g2.Vb * nv1;
    cx<double>* HP = reinterpret_cast<cx<double>*>(smem_l2);          // [nc1][nc2]
    cx<double>* PX = HP + (size_t)nc1 * nc2;                           // [nc2][nv1]
    const int X2 = blockIdx.x / 9, d = blockIdx.x - X2 * 9;
    const int ne = nc2 * nc2;
    cx<double> acc[kL2MaxEntries];
#pragma unroll
    for (int q = 0; q < kL2MaxEntries; ++q) acc[q] = cx<double>(0, 0);
    for (int l2 = 0; l2 < g2.Vb; ++l2) {
        int lc[4];
        local_coords(g2, l2, lc);
        const int X1 = (int)lex_site(g2, X2, l2);
        for (int t = 0; t < 9; ++t) {
            int slot = 0;
            if (t > 0) {
                const int mu = (t - 1) >> 1;
                const bool fwd = (t & 1) != 0;
                const bool leaves = fwd ? (lc[mu] == g2.B[mu] - 1) : (lc[mu] == 0);
                slot = leaves ? t : 0;
            }
            if (slot != d) continue;
            const int Y1 = coarse_neighbour(g1, X1, t);
            int Y2, ly2;
            level1_to_level2(g2, Y1, Y2, ly2);
            __syncthreads();
            // rows of P2 at x: PX[a][j] = P2 column a on dof s_a Nv1 + j at (X2, l2)
            for (int e = threadIdx.x; e < nc2 * nv1; e += blockDim.x) {
                const int a = e / nv1, j = e - a * nv1, sa = a / nv2, ia = a - sa * nv2;
                PX[e] = ld<double>(P2 + (((size_t)X2 * 2 + sa) * nv2 + ia) * len + (size_t)l2 * nv1 + j);
            }
            // HP[q][b] = sum_j A1[X1][t](q, s_b Nv1 + j) P2 column b at (Y2, ly2)
            const double2* At = A1 + ((size_t)X1 * 9 + t) * nc1 * nc1;
            for (int e = threadIdx.x; e < nc1 * nc2; e += blockDim.x) {
                const int q = e / nc2, b = e - q * nc2, sb = b / nv2, ib = b - sb * nv2;
                const double2* pb = P2 + (((size_t)Y2 * 2 + sb) * nv2 + ib) * len + (size_t)ly2 * nv1;
                cx<double> h(0, 0);
                for (int j = 0; j < nv1; ++j)
                    cmad(h, ld<double>(At + (size_t)(sb * nv1 + j) * nc1 + q), ld<double>(pb + j));
                HP[e] = h;
            }
            __syncthreads();
#pragma unroll
            for (int qq = 0; qq < kL2MaxEntries; ++qq) {
                const int e = threadIdx.x + qq * blockDim.x;
                if (e < ne) {
                    const int a = e / nc2, b = e - a * nc2, sa = a / nv2;
                    for (int j = 0; j < nv1; ++j) cmadc(acc[qq], PX[a * nv1 + j], HP[(size_t)(sa * nv1 + j) * nc2 + b]);
                }
            }
        }
    }
#pragma unroll
    for (int qq = 0; qq < kL2MaxEntries; ++qq) {
        const int e = threadIdx.x + qq * blockDim.x;
        if (e < ne) {
            const int a = e / nc2, b = e - a * nc2;
            st<double>(A2 + (((size_t)X2 * 9 + d) * nc2 + b) * nc2 + a, acc[qq]);
        }
    }
}

// ---------------------------------------------------------------- launchers
void block_orthonormalize_l2(double2* P2, const double2* V2, int nv1, int nv2, const Geom& g2, int* status,
                             cudaStream_t st) {
    note_launch();
    k_block_ortho_l2<<<2 * g2.Vc, kL2Threads, 0, st>>>(P2, V2, nv1, nv2, g2, status);
}
template <typename T>
void restrict_l2(v2<T>* r2, const v2<T>* P2, const v2<T>* r1, int nv1, int nv2, const Geom& g2, cudaStream_t st) {
    note_launch();
    k_restrict_l2<T><<<g2.Vc, kL2Threads, 0, st>>>(r2, P2, r1, nv1, nv2, g2);
}
template <typename T>
void prolong_l2(v2<T>* e1, const v2<T>* P2, const v2<T>* y2, int nv1, int nv2, const Geom& g2, cudaStream_t st) {
    const long long n = g2.V * 2LL * nv1;
    note_launch();
    k_prolong_l2<T><<<(int)((n + kL2Threads - 1) / kL2Threads), kL2Threads, 0, st>>>(e1, P2, y2, nv1, nv2, g2);
}
size_t build_l2_smem(int nv1, int nv2) { return sizeof(cx<double>) * ((size_t)4 * nv1 * nv2 + (size_t)2 * nv2 * nv1); }
bool build_l2_supported(int nv1, int nv2) {
    return 4 * nv2 * nv2 <= kL2MaxEntries * kL2Threads && build_l2_smem(nv1, nv2) <= 200 * 1024;
}
cudaError_t coarse_build_l2(double2* A2, const double2* P2, const double2* A1, int nv1, int nv2, const Geom& g1,
                            const Geom& g2, cudaStream_t st) {
    if (!build_l2_supported(nv1, nv2)) return cudaErrorInvalidValue;
    const size_t sm = build_l2_smem(nv1, nv2);
    cudaError_t e = cudaFuncSetAttribute(k_build_l2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    note_launch();
    k_build_l2<<<g2.Vc * 9, kL2Threads, sm, st>>>(A2, P2, A1, nv1, nv2, g1, g2);
    return cudaGetLastError();
}
template void restrict_l2<float>(v2<float>*, const v2<float>*, const v2<float>*, int, int, const Geom&, cudaStream_t);
template void restrict_l2<double>(v2<double>*, const v2<double>*, const v2<double>*, int, int, const Geom&,
                                  cudaStream_t);
template void prolong_l2<float>(v2<float>*, const v2<float>*, const v2<float>*, int, int, const Geom&, cudaStream_t);
template void prolong_l2<double>(v2<double>*, const v2<double>*, const v2<double>*, int, int, const Geom&,
                                 cudaStream_t);

}  // namespace wmg

// Batched (multi right-hand side) coarse level: the coarse stencil applied to
// an RHS panel on the 5th-generation tensor cores, and the per-RHS CGNR steps.
//
// Panel layout: xB[X][b][n] complex FP32, n < npad (RHS index fastest, npad a
// multiple of 16).  For one aggregate X the stencil is a dense contraction
//   y[X][a][n] = sum_d sum_b A[X][d][a][b] x[X+d][b][n],
// written as a real GEMM through the embedding
//   [Re y]   [Re A  -Im A] [Re x]
//   [Im y] = [Im A   Re A] [Im x]      (M = K = 2 nc per direction d),
// M padded to 128, K = 9 * 2nc, N = npad.  A is stored once per (X, d) in
// FP16 in the tensor-core shared-memory layout and copied with the bulk-copy
// engine; x is split into FP16 hi + lo parts (x = hi + lo to ~22 bits) so two
// MMAs per K step give an FP32-accurate product against the FP16 operator.
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "mg_launch.h"
#include "mg_ptx.cuh"

namespace wmg {

// half offset of element (row r, k) in a K-major core-matrix tile with K columns
__host__ __device__ __forceinline__ int core_off(int r, int k, int K) {
    return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

// ---------------------------------------------------------------- operator embedding
// Aemb[X][d]: 2nc x 2nc FP16 real embedding of A[X][d] in the core-matrix layout
// (rows 2nc..127 of the 128-row MMA tile are zero in shared memory only).
__global__ void k_coarse_embed(__half* Aemb, const double2* __restrict__ A, int nc, long long nblk) {
    const int K = 2 * nc;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = nblk * K * K;
    if (idx >= total) return;
    long long blk = idx / (K * K);
    int rem = (int)(idx - blk * K * K);
    int m = rem / K, k = rem - m * K;
    int a = m % nc, b = k % nc;
    bool imr = m >= nc, imc = k >= nc;
    double2 v = A[blk * nc * nc + (size_t)b * nc + a];   // column-major block: A[b][a] = A_ab
    double e = (!imr && !imc) ? v.x : (!imr && imc) ? -v.y : (imr && !imc) ? v.y : v.x;
    Aemb[blk * K * K + core_off(m, k, K)] = __double2half(e);
}

void coarse_embed(__half* Aemb, const double2* A, int nc, int Vc, cudaStream_t st) {
    long long nblk = (long long)Vc * 9;
    long long total = nblk * 4 * nc * nc;
    note_launch();
    k_coarse_embed<<<(int)((total + 255) / 256), 256, 0, st>>>(Aemb, A, nc, nblk);
}

// ---------------------------------------------------------------- tensor-core batched stencil
constexpr int kTcThreads = 128;
constexpr int kTcMaxStages = 3;   // pipeline depth when it fits shared memory, else 2
constexpr long long kTcWaitLimit = 20000000LL;

__host__ __device__ inline int tc_tmem_cols(int npad) {
    int c = 32;
    while (c < npad) c <<= 1;
    return c;
}
// one pipeline stage: the (padded) 128-row A tile, the hi and lo B tiles
__host__ __device__ inline size_t tc_stage_bytes(int nc, int nw) {
    const size_t K = 2 * nc;
    return 128 * K * 2 + 2 * (size_t)nw * K * 2;
}
constexpr size_t kTcStaticSmem = 256;   // barriers, TMEM address, flag
__host__ __device__ inline int tc_stages(int nc, int nw) {
    return kTcMaxStages * tc_stage_bytes(nc, nw) + kTcStaticSmem <= 227 * 1024 ? kTcMaxStages : 2;
}
__host__ __device__ inline int tc_stages_of(const TcApplyArgs& a) { return a.stages > 0 ? a.stages : tc_stages(a.nc, a.nw); }

// The operand panel as FP16 hi + lo tiles in the tensor-core shared-memory
// layout, one tile pair per (aggregate Y, column chunk c):
//   bt[((Y * nch + c) * 2 + {0 hi, 1 lo}) * nw * K + core_off(n, k, K)],
// k = b (real part) or nc + b (imaginary part) of x[Y][b][c * nw + n], with the
// column scale and, for the adjoint, the sigma3 sign of rows b >= nc/2 applied.
// One thread per (Y, c, n, 8-column group of k): two 16-byte stores.
__global__ void k_tc_split(__half* __restrict__ bt, const float2* __restrict__ x, int nc, int npad, int nw, int dag,
                           const double* __restrict__ colscale, long long total) {
    const int K = 2 * nc, kg8 = K >> 3, nch = npad / nw, nvh = nc >> 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int kg = (int)(i % kg8);
        long long t = i / kg8;
        const int n = (int)(t % nw);
        t /= nw;
        const int c = (int)(t % nch);
        const long long Y = t / nch;
        const int col = c * nw + n;
        const float sc = colscale ? (float)colscale[col] : 1.f;
        __align__(16) __half hi[8], lo[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = kg * 8 + e, b = k < nc ? k : k - nc;
            const float2 v = x[((size_t)Y * nc + b) * npad + col];
            float f = (k < nc ? v.x : v.y) * sc;
            if (dag && b >= nvh) f = -f;
            const __half h = __float2half_rn(f);
            hi[e] = h;
            lo[e] = __float2half_rn(f - __half2float(h));
        }
        __half* base = bt + ((size_t)(Y * nch + c) * 2) * nw * K + core_off(n, kg * 8, K);
        *reinterpret_cast<uint4*>(base) = *reinterpret_cast<const uint4*>(hi);
        *reinterpret_cast<uint4*>(base + (size_t)nw * K) = *reinterpret_cast<const uint4*>(lo);
    }
}

// One CTA per (aggregate X, column chunk of width nw).  Thread 0 runs a
// pipeline of 3 (or, where shared memory is short, 2) stages over the 9
// directions d: the bulk-copy engine brings
// A_emb[X][d] and the hi/lo tiles of x[X+d] (split beforehand by k_tc_split)
// into a stage, thread 0 issues the MMAs (hi and lo per K step) into the TMEM
// accumulator (128 lanes = embedded rows, nw columns = right-hand sides) and
// commits them to the stage's "empty" barrier; a stage is refilled once its
// MMAs are done.  Then the four warps read the accumulator back.
__global__ void __launch_bounds__(kTcThreads, 1) k_coarse_apply_tc(TcApplyArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    // grid (column chunks, aggregates): the chunks of one aggregate run side by
    // side and share its operator tiles through L2
    const int nc = a.nc, npad = a.npad, nw = a.nw, chunk = blockIdx.x, n0 = chunk * nw, K = 2 * nc, nvh = nc / 2;
    const int nch = npad / nw, S = tc_stages_of(a);
    const size_t SA = (size_t)128 * K * 2, SB = (size_t)nw * K * 2, SS = SA + 2 * SB;
    __shared__ __align__(8) uint64_t bar[2 * kTcMaxStages];   // [0, S): stage full, [S, 2S): stage empty
    __shared__ uint32_t s_taddr;
    __shared__ int s_ok;
    const int X = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = tc_tmem_cols(nw);
    const uint32_t bytesA = (uint32_t)(K * K * 2), bytesB = (uint32_t)SB;

    if (tid == 0) {
        for (int i = 0; i < 2 * S; ++i) mbar_init(bar + i, 1);
        fence_mbar_init();
    }
    // zero the padding rows (2nc..127) of every stage's A tile once
    for (int st = 0; st < S; ++st) {
        __half* As = reinterpret_cast<__half*>(smem + st * SS);
        for (int i = K * K + tid; i < 128 * K; i += kTcThreads) As[i] = __float2half(0.f);
    }
    fence_proxy_async();   // the zeros are read by the MMAs (async proxy)
    if (warp == 0) {
        tmem_alloc(&s_taddr, ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_taddr;

    if (tid == 0) {
        const uint32_t idesc = idesc_f16(128, nw);
        const uint32_t lbo = 128, sbo = (uint32_t)(K >> 3) * 128;
        // stage bookkeeping for the drain: parity of the copy in flight per stage (-1: none)
        int pending[kTcMaxStages];
        for (int st = 0; st < kTcMaxStages; ++st) pending[st] = -1;
        auto issue = [&](int d, int st) {
            unsigned char* base = smem + st * SS;
            const int Y = coarse_neighbour(a.g, X, d);
            mbar_expect_tx(bar + st, bytesA + 2 * bytesB);
            bulk_copy_g2s(base, a.Aemb + ((size_t)X * 9 + d) * K * K, bytesA, bar + st);
            const __half* bsrc = a.bt + ((size_t)(Y * nch + chunk) * 2) * nw * K;
            bulk_copy_g2s(base + SA, bsrc, bytesB, bar + st);
            bulk_copy_g2s(base + SA + SB, bsrc + (size_t)nw * K, bytesB, bar + st);
            pending[st] = (d / S) & 1;
        };
        bool ok = true;
        int last = -1;   // stage * 2 + parity of the last commit
        for (int d = 0; d < S && d < 9; ++d) issue(d, d);
        for (int d = 0; d < 9 && ok; ++d) {
            // refill the stage the previous direction's MMAs used, once they are done
            const int dp = d - 1;
            if (dp >= 0 && dp + S < 9) {
                const int sp = dp % S;
                if (!mbar_wait(bar + S + sp, (uint32_t)((dp / S) & 1), kTcWaitLimit)) { ok = false; break; }
                issue(dp + S, sp);
            }
            const int s = d % S;
            if (!mbar_wait(bar + s, (uint32_t)((d / S) & 1), kTcWaitLimit)) { ok = false; break; }
            pending[s] = -1;
            tc_fence_after();
            const uint32_t a0 = smem_u32(smem + s * SS), bh0 = a0 + (uint32_t)SA, bl0 = bh0 + (uint32_t)SB;
            for (int ks = 0; ks < (K >> 4); ++ks) {
                const uint64_t ad = smem_desc(a0 + ks * 256, lbo, sbo);
                mma_f16(tmem, ad, smem_desc(bh0 + ks * 256, lbo, sbo), idesc, (d > 0 || ks > 0) ? 1u : 0u);
                mma_f16(tmem, ad, smem_desc(bl0 + ks * 256, lbo, sbo), idesc, 1u);
            }
            mma_commit(bar + S + s);
            last = s * 2 + ((d / S) & 1);
        }
        // drain: the last commit covers every MMA issued; then every copy still in flight
        if (last >= 0 && !mbar_wait(bar + S + (last >> 1), (uint32_t)(last & 1), kTcWaitLimit)) ok = false;
        for (int st = 0; st < S; ++st)
            if (pending[st] >= 0 && !mbar_wait(bar + st, (uint32_t)pending[st], kTcWaitLimit)) ok = false;
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    const bool ok = s_ok != 0;
    tc_fence_after();
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (embedded rows m) into a
    // row-major tile in the (now idle) stage memory, T[m][n] (stride nw + 1);
    // then rows a (real part) and nc + a (imaginary part) leave as one complex
    // column-contiguous row of y, coalesced over the right-hand sides n
    float* T = reinterpret_cast<float*>(smem);
    const int ts = nw + 1;
    const int m = warp * 32 + lane;
    for (int c0 = 0; c0 < nw; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (m < K)
#pragma unroll
            for (int j = 0; j < 16; ++j)
                T[m * ts + c0 + j] = a.colscale ? v[j] * (float)(1.0 / a.colscale[n0 + c0 + j]) : v[j];
    }
    tc_fence_before();
    __syncthreads();
    if (ok) {
        float2* y = a.y;
        for (int i = tid; i < nc * nw; i += kTcThreads) {
            const int ar = i / nw, n = i - ar * nw;
            const float sg = (a.dag && ar >= nvh) ? -1.f : 1.f;
            y[((size_t)X * nc + ar) * npad + n0 + n] = make_float2(sg * T[ar * ts + n], sg * T[(nc + ar) * ts + n]);
        }
        if (a.norms)
            for (int n = tid; n < nw; n += kTcThreads) {
                float q = 0.f;
                for (int r = 0; r < K; ++r) q += T[r * ts + n] * T[r * ts + n];
                a.norms[(size_t)X * npad + n0 + n] = q;
            }
    } else if (a.norms) {
        for (int n = tid; n < nw; n += kTcThreads) a.norms[(size_t)X * npad + n0 + n] = 0.f;
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// Dynamic shared memory of one CTA: its pipeline stages, padded so that at
// most 512 / ncols CTAs fit on an SM (their TMEM allocations never exceed the
// 512 columns of an SM, so no allocation waits).
static size_t tc_launch_smem(int nc, int nw, int stages) {
    size_t sm = (size_t)stages * tc_stage_bytes(nc, nw);
    size_t per_sm = 228 * 1024, cap = 512 / tc_tmem_cols(nw);
    size_t min_sm = per_sm / (cap + 1) + 1024;
    return sm > min_sm ? sm : min_sm;
}
bool coarse_apply_tc_supported(int nc, int npad) {
    return npad % 16 == 0 && npad >= 16 && npad <= 256 && (2 * nc) % 16 == 0 && 2 * nc <= 128 &&
           tc_launch_smem(nc, npad, 2) + kTcStaticSmem <= 227 * 1024;
}
// attribute for the largest chunk width used with this nc (every nw <= npad fits)
cudaError_t coarse_apply_tc_prepare(int nc, int npad) {
    if (!coarse_apply_tc_supported(nc, npad)) return cudaErrorInvalidValue;
    size_t mx = 0;
    for (int nw = 16; nw <= npad; nw += 16) mx = std::max(mx, tc_launch_smem(nc, nw, tc_stages(nc, nw)));
    return cudaFuncSetAttribute(k_coarse_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
}
// launch only (coarse_apply_tc_prepare must have been called for this shape);
// args.nw = column chunk per CTA (multiple of 16 dividing npad; 0 = npad)
cudaError_t coarse_apply_tc(const TcApplyArgs& args, cudaStream_t st) {
    TcApplyArgs a = args;
    if (a.nw <= 0) a.nw = a.npad;
    if (!a.bt || a.g.Vc > 65535) return cudaErrorInvalidValue;   // aggregates index grid.y
    const long long total = (long long)a.g.Vc * a.npad * (2 * a.nc / 8);
    note_launch();
    k_tc_split<<<(int)std::min<long long>((total + 255) / 256, 16LL * device_sm_count()), 256, 0, st>>>(
        a.bt, a.x, a.nc, a.npad, a.nw, a.dag, a.colscale, total);
    TmemOrder order(st);
    if (order.error() != cudaSuccess) return order.error();
    note_launch();
    if (a.stages != 0 && (a.stages < 2 || a.stages > tc_stages(a.nc, a.nw))) return cudaErrorInvalidValue;
    k_coarse_apply_tc<<<dim3(a.npad / a.nw, a.g.Vc), kTcThreads, tc_launch_smem(a.nc, a.nw, tc_stages_of(a)), st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return order.launched();
}

// Chunk width and pipeline depth for (nc, npad): every candidate (multiples of
// 16 dividing npad; 2 or 3 stages where 3 fit -- 2 can leave room for a second
// CTA on the SM) is timed with CUDA events on the given stream and the fastest
// is kept.  The cache is keyed by device as well and guarded for concurrent
// host threads.
int coarse_apply_tc_tune(const TcApplyArgs& args, cudaStream_t st, int* stages) {
    struct Entry { int dev, nc, npad, nw, stages; };
    static std::vector<Entry> cache;
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry& e : cache)
            if (e.dev == dev && e.nc == args.nc && e.npad == args.npad) {
                if (stages) *stages = e.stages;
                return e.nw;
            }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = args.npad, best_s = tc_stages(args.nc, args.npad);
    float best_ms = 1e30f;
    for (int cand = 0; cand < 2 * 16; ++cand) {
        const int nw = 16 * (cand / 2 + 1), S = 2 + cand % 2;
        if (nw > args.npad || args.npad % nw || S > tc_stages(args.nc, nw)) continue;
        TcApplyArgs a = args;
        a.nw = nw;
        a.stages = S;
        coarse_apply_tc(a, st);   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5; ++r) coarse_apply_tc(a, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = nw; best_s = S; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lock(mu);
    cache.push_back({dev, args.nc, args.npad, best, best_s});
    if (stages) *stages = best_s;
    return best;
}

// ---------------------------------------------------------------- SIMT reference of the same contraction
// One thread per (X, a, n); reads the FP64 operator.  Used by the FP64 batched
// path and to cross-check the tensor-core kernel.
template <typename T>
__global__ void k_coarse_apply_batched_simt(v2<T>* __restrict__ y, const double2* __restrict__ A,
                                            const v2<T>* __restrict__ x, int nc, int npad, int dag, Geom g,
                                            float* norms) {
    int X = blockIdx.x, a = blockIdx.y;
    int nvh = nc / 2;
    for (int n = threadIdx.x; n < npad; n += blockDim.x) {
        cx<double> acc(0, 0);
        for (int d = 0; d < 9; ++d) {
            int Y = coarse_neighbour(g, X, d);
            const double2* Ad = A + ((size_t)X * 9 + d) * nc * nc + a;
            for (int b = 0; b < nc; ++b) {
                v2<T> xv = x[((size_t)Y * nc + b) * npad + n];
                cx<double> xb((double)xv.x, (double)xv.y);
                if (dag && b >= nvh) xb = cx<double>(-xb.r, -xb.i);
                cmad(acc, ld<double>(Ad + (size_t)b * nc), xb);
            }
        }
        if (dag && a >= nvh) acc = cx<double>(-acc.r, -acc.i);
        v2<T> o; o.x = (T)acc.r; o.y = (T)acc.i;
        y[((size_t)X * nc + a) * npad + n] = o;
    }
    (void)norms;
}
template <typename T>
void coarse_apply_batched_simt(v2<T>* y, const double2* A, const v2<T>* x, int nc, int npad, bool dag, const Geom& g,
                               cudaStream_t st) {
    note_launch();
    k_coarse_apply_batched_simt<T><<<dim3(g.Vc, nc), 128, 0, st>>>(y, A, x, nc, npad, dag ? 1 : 0, g, nullptr);
}
template void coarse_apply_batched_simt<float>(v2<float>*, const double2*, const v2<float>*, int, int, bool,
                                               const Geom&, cudaStream_t);
template void coarse_apply_batched_simt<double>(v2<double>*, const double2*, const v2<double>*, int, int, bool,
                                                const Geom&, cudaStream_t);

// ---------------------------------------------------------------- per-RHS CGNR steps
// Per-RHS scalars (double, npad entries each) in BatchScal.  Column sums are
// reduced in two fixed-order stages: per-block partials part[block][n], then
// one CTA per column adds the partials.  Columns whose done flag is set are
// frozen.
constexpr int kRowChunks = kBatchRowChunks;

// rows [r0, r1) of block b of nb over `rows`; thread (rg, n), rgs row groups
struct ColTile {
    int n, rg, rgs;
    long long r0, r1;
    __device__ ColTile(int npad, long long rows) {
        rgs = blockDim.x / npad;
        if (rgs < 1) rgs = 1;
        n = threadIdx.x % npad;
        rg = threadIdx.x / npad;
        r0 = (long long)blockIdx.x * rows / gridDim.x;
        r1 = (long long)(blockIdx.x + 1) * rows / gridDim.x;
    }
    __device__ bool active() const { return rg < rgs; }
};
// per-column sum of v over the row groups of this block (fixed order) -> part[blockIdx][n]
__device__ __forceinline__ void col_partial(float v, const ColTile& t, int npad, float* sh, float* part) {
    if (t.active()) sh[t.rg * npad + t.n] = v;
    __syncthreads();
    for (int n = threadIdx.x; n < npad; n += blockDim.x) {
        float s = 0.f;
        for (int g = 0; g < t.rgs; ++g) s += sh[g * npad + n];
        part[(size_t)blockIdx.x * npad + n] = s;
    }
}
// one CTA per column: sum of part[c][n] over c < nparts, fixed order
__device__ __forceinline__ double col_total(const float* part, int nparts, int npad) {
    __shared__ double sh[33];
    const int n = blockIdx.x;
    double a = 0;
    for (int c = threadIdx.x; c < nparts; c += blockDim.x) a += (double)part[(size_t)c * npad + n];
    double v[1] = {a};
    block_reduce<1>(v, (double (*)[32])sh);
    if (threadIdx.x == 0) sh[32] = v[0];
    __syncthreads();
    return sh[32];
}

__global__ void k_bcol_norm(const float2* __restrict__ v, long long rows, int npad, float* part) {
    extern __shared__ float shf[];
    ColTile t(npad, rows);
    float s = 0.f;
    if (t.active())
        for (long long r = t.r0 + t.rg; r < t.r1; r += t.rgs) {
            float2 a = v[r * npad + t.n];
            s += a.x * a.x + a.y * a.y;
        }
    col_partial(s, t, npad, shf, part);
}
// scale_n = ||rc_n||, done = (scale == 0 || n >= nrhs)
// power of two nearest sqrt(rows / s): entries of a column with |x|^2 = s then sit
// near 1 in magnitude, far above the FP16 subnormal range, after scaling
__device__ __forceinline__ double pow2_scale(double s, long long rows) {
    if (!(s > 0)) return 1.0;
    const double e = rint(0.5 * log2((double)rows / s));
    return exp2(fmin(fmax(e, -120.0), 120.0));
}
__global__ void k_bcg_scale(BatchScal S, const float* part, int nparts, int npad, int nrhs, int maxit, long long rows) {
    double s = col_total(part, nparts, npad);
    if (threadIdx.x != 0) return;
    int n = blockIdx.x;
    double sc = sqrt(s);
    S.scale[n] = sc;
    S.done[n] = (n >= nrhs || !(sc > 0) || maxit <= 0) ? 1.0 : 0.0;
    S.iters[n] = 0;
    S.r2[n] = S.done[n] != 0 ? 0.0 : 1.0;
    S.csr[n] = pow2_scale(1.0, rows);   // r starts with unit norm
}
__global__ void k_bcg_start(float2* __restrict__ y, float2* __restrict__ r, const float2* __restrict__ rc,
                            long long total, int npad, BatchScal S) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int n = (int)(i % npad);
        double sc = S.scale[n];
        float f = sc > 0 ? (float)(1.0 / sc) : 0.f;
        float2 v = rc[i];
        r[i] = make_float2(v.x * f, v.y * f);
        y[i] = make_float2(0.f, 0.f);
    }
}
// gamma = ||s||^2 (first direction)
__global__ void k_bcg_gamma0(BatchScal S, const float* xpart, int nx, int npad, long long rows) {
    double s = col_total(xpart, nx, npad);
    if (threadIdx.x == 0) {
        S.gamma[blockIdx.x] = s;
        S.csp[blockIdx.x] = pow2_scale(s, rows);   // p = s
    }
}
// alpha = gamma / ||q||^2
__global__ void k_bcg_alpha(BatchScal S, const float* xpart, int nx, int npad) {
    double s = col_total(xpart, nx, npad);
    int n = blockIdx.x;
    if (threadIdx.x != 0 || S.done[n] != 0) return;
    if (s > 0) S.alpha[n] = S.gamma[n] / s;
    else { S.alpha[n] = 0; S.done[n] = 1; }
}
// y += alpha p, r -= alpha q (active columns), column partials of ||r||^2; zeroes *active
__global__ void k_bcg_update1(float2* __restrict__ y, float2* __restrict__ r, const float2* __restrict__ p,
                              const float2* __restrict__ q, long long rows, int npad, BatchScal S, float* part,
                              int* active) {
    extern __shared__ float shf[];
    if (blockIdx.x == 0 && threadIdx.x == 0) *active = 0;
    ColTile t(npad, rows);
    float s = 0.f;
    if (t.active() && S.done[t.n] == 0) {
        const float al = (float)S.alpha[t.n];
        for (long long rr = t.r0 + t.rg; rr < t.r1; rr += t.rgs) {
            long long i = rr * npad + t.n;
            float2 pv = p[i], qv = q[i], yv = y[i], rv = r[i];
            y[i] = make_float2(yv.x + al * pv.x, yv.y + al * pv.y);
            float2 rn = make_float2(rv.x - al * qv.x, rv.y - al * qv.y);
            r[i] = rn;
            s += rn.x * rn.x + rn.y * rn.y;
        }
    }
    col_partial(s, t, npad, shf, part);
}
// ||r||^2, iteration count, stopping test; *active counts columns still running
__global__ void k_bcg_check(BatchScal S, const float* part, int nparts, int npad, double tol2, int maxit, int* active,
                            long long rows) {
    double s = col_total(part, nparts, npad);
    int n = blockIdx.x;
    if (threadIdx.x != 0 || S.done[n] != 0) return;
    S.r2[n] = s;                         // relative to ||rc_n||^2 = 1 after scaling
    S.csr[n] = pow2_scale(s, rows);
    S.iters[n] += 1;
    if (s <= tol2 || S.iters[n] >= maxit) S.done[n] = 1;
    else atomicAdd(active, 1);
}
// beta = ||s||^2 / gamma, gamma = ||s||^2
__global__ void k_bcg_beta(BatchScal S, const float* xpart, int nx, int npad, long long rows) {
    double s = col_total(xpart, nx, npad);
    int n = blockIdx.x;
    if (threadIdx.x != 0 || S.done[n] != 0) return;
    S.beta[n] = S.gamma[n] > 0 ? s / S.gamma[n] : 0.0;
    S.gamma[n] = s;
    S.csp[n] = pow2_scale(s, rows);      // p = s + beta p is of the size of s or larger
}
__global__ void k_bcg_update2(float2* __restrict__ p, const float2* __restrict__ s, long long total, int npad,
                              BatchScal S, int first) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int n = (int)(i % npad);
        if (!first && S.done[n] != 0) continue;
        float be = first ? 0.f : (float)S.beta[n];
        float2 sv = s[i], pv = first ? make_float2(0.f, 0.f) : p[i];
        p[i] = make_float2(sv.x + be * pv.x, sv.y + be * pv.y);
    }
}
// y *= scale (undo the normalisation)
__global__ void k_bcg_unscale(float2* __restrict__ y, long long total, int npad, BatchScal S) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int n = (int)(i % npad);
        float f = (float)S.scale[n];
        float2 v = y[i];
        y[i] = make_float2(v.x * f, v.y * f);
    }
}

static inline int ew_grid(long long total) {
    long long b = (total + 255) / 256;
    if (b > 8LL * device_sm_count()) b = 8LL * device_sm_count();
    return (int)(b > 0 ? b : 1);
}
static inline int col_threads(int npad) {
    int rgs = 256 / npad;
    if (rgs < 1) rgs = 1;
    return ((rgs * npad + 31) / 32) * 32;
}
static inline size_t col_smem(int npad) { return sizeof(float) * (size_t)col_threads(npad) + sizeof(float) * npad; }

// One CGLS iteration on all columns (kernels only: capturable in a CUDA graph).
void bcg_iteration(const BatchCg& c, cudaStream_t st) {
    const long long rows = (long long)c.g.Vc * c.nc, total = rows * c.npad;
    const int ct = col_threads(c.npad);
    const size_t cs = col_smem(c.npad);
    TcApplyArgs ap{c.Aemb, c.p, c.q, c.nc, c.npad, c.nw, 0, c.g, c.xpart, c.err, c.S.csp, c.bt, c.stages};
    coarse_apply_tc(ap, st);                                                               // q = D_c p
    note_launch();
    k_bcg_alpha<<<c.npad, 256, 0, st>>>(c.S, c.xpart, c.g.Vc, c.npad);
    note_launch();
    k_bcg_update1<<<kRowChunks, ct, cs, st>>>(c.y, c.r, c.p, c.q, rows, c.npad, c.S, c.rpart, c.active);
    note_launch();
    k_bcg_check<<<c.npad, 256, 0, st>>>(c.S, c.rpart, kRowChunks, c.npad, c.tol2, c.maxit, c.active, rows);
    TcApplyArgs as{c.Aemb, c.r, c.s, c.nc, c.npad, c.nw, 1, c.g, c.xpart, c.err, c.S.csr, c.bt, c.stages};
    coarse_apply_tc(as, st);                                                               // s = D_c^dag r
    note_launch();
    k_bcg_beta<<<c.npad, 256, 0, st>>>(c.S, c.xpart, c.g.Vc, c.npad, rows);
    note_launch();
    k_bcg_update2<<<ew_grid(total), 256, 0, st>>>(c.p, c.s, total, c.npad, c.S, 0);
}

// y = 0, r = rc/||rc||, s = D_c^dag r, gamma, p = s
void bcg_start(const BatchCg& c, cudaStream_t st) {
    const long long rows = (long long)c.g.Vc * c.nc, total = rows * c.npad;
    note_launch();
    k_bcol_norm<<<kRowChunks, col_threads(c.npad), col_smem(c.npad), st>>>(c.rc, rows, c.npad, c.rpart);
    note_launch();
    k_bcg_scale<<<c.npad, 256, 0, st>>>(c.S, c.rpart, kRowChunks, c.npad, c.nrhs, c.maxit, rows);
    note_launch();
    k_bcg_start<<<ew_grid(total), 256, 0, st>>>(c.y, c.r, c.rc, total, c.npad, c.S);
    TcApplyArgs as{c.Aemb, c.r, c.s, c.nc, c.npad, c.nw, 1, c.g, c.xpart, c.err, c.S.csr, c.bt, c.stages};
    coarse_apply_tc(as, st);
    note_launch();
    k_bcg_gamma0<<<c.npad, 256, 0, st>>>(c.S, c.xpart, c.g.Vc, c.npad, rows);
    note_launch();
    k_bcg_update2<<<ew_grid(total), 256, 0, st>>>(c.p, c.s, total, c.npad, c.S, 1);
}

void bcg_finish(const BatchCg& c, cudaStream_t st) {
    const long long total = (long long)c.g.Vc * c.nc * c.npad;
    note_launch();
    k_bcg_unscale<<<ew_grid(total), 256, 0, st>>>(c.y, total, c.npad, c.S);
}

}  // namespace wmg

namespace wmg {
static inline int ew_grid2(long long total) {
    long long b = (total + 255) / 256;
    if (b > 8LL * device_sm_count()) b = 8LL * device_sm_count();
    return (int)(b > 0 ? b : 1);
}
// columns n < nrhs of a panel from nrhs stacked coarse vectors in[n][row] (FP64), other columns zero
__global__ void k_panel_pack(float2* __restrict__ out, const double2* __restrict__ in, long long rows, int nrhs, int npad) {
    long long total = rows * npad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long r = i / npad;
        int n = (int)(i - r * npad);
        float2 v = make_float2(0.f, 0.f);
        if (n < nrhs) {
            double2 d = in[(size_t)n * rows + r];
            v = make_float2((float)d.x, (float)d.y);
        }
        out[i] = v;
    }
}
__global__ void k_panel_unpack(double2* __restrict__ out, const float2* __restrict__ in, long long rows, int nrhs, int npad) {
    long long total = rows * nrhs;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long n = i / rows, r = i - n * rows;
        float2 v = in[r * npad + n];
        out[i] = make_double2((double)v.x, (double)v.y);
    }
}
template <typename T>
__global__ void k_panel_pack_t(v2<T>* __restrict__ out, const double2* __restrict__ in, long long rows, int nrhs, int npad) {
    long long total = rows * npad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long r = i / npad;
        int n = (int)(i - r * npad);
        v2<T> v; v.x = 0; v.y = 0;
        if (n < nrhs) { double2 d = in[(size_t)n * rows + r]; v.x = (T)d.x; v.y = (T)d.y; }
        out[i] = v;
    }
}
template <typename T>
__global__ void k_panel_unpack_t(double2* __restrict__ out, const v2<T>* __restrict__ in, long long rows, int nrhs, int npad) {
    long long total = rows * nrhs;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long n = i / rows, r = i - n * rows;
        v2<T> v = in[r * npad + n];
        out[i] = make_double2((double)v.x, (double)v.y);
    }
}
void panel_pack(float2* out, const double2* in, long long rows, int nrhs, int npad, cudaStream_t st) {
    note_launch();
    k_panel_pack<<<ew_grid2(rows * npad), 256, 0, st>>>(out, in, rows, nrhs, npad);
}
void panel_unpack(double2* out, const float2* in, long long rows, int nrhs, int npad, cudaStream_t st) {
    note_launch();
    k_panel_unpack<<<ew_grid2(rows * nrhs), 256, 0, st>>>(out, in, rows, nrhs, npad);
}
void panel_pack64(double2* out, const double2* in, long long rows, int nrhs, int npad, cudaStream_t st) {
    note_launch();
    k_panel_pack_t<double><<<ew_grid2(rows * npad), 256, 0, st>>>(out, in, rows, nrhs, npad);
}
void panel_unpack64(double2* out, const double2* in, long long rows, int nrhs, int npad, cudaStream_t st) {
    note_launch();
    k_panel_unpack_t<double><<<ew_grid2(rows * nrhs), 256, 0, st>>>(out, in, rows, nrhs, npad);
}
}  // namespace wmg

// Coarse CGNR (CGLS, Sec. IV: CG on the normal equations of D_c) in one
// persistent cooperative launch, with the coarse operator held on chip.
//
// Work split.  The operator rows of every aggregate X are cut into H = nc/RU
// chunks of RU rows; a "unit" u = X*H + h holds rows h*RU .. h*RU+RU-1 of all
// nine blocks of X and is stored contiguously,
//     Au[u][d 9][b nc][a RU]        (FP32 complex, or FP16 complex + su[X][d])
// so one bulk copy moves it.  CTA c (one per SM) owns the contiguous range of
// units [c*NU/G, (c+1)*NU/G); the owner of unit (X, h) computes output rows
// h*RU.. of X and does the elementwise CG updates of those entries, so every
// entry is written by exactly one CTA.
//
// On-chip operator.  When a CTA's units fit in shared memory they are copied
// once per launch and stay there for all iterations ("resident"); otherwise
// they stream through a ring of slot groups, and the copies for the next
// phase are issued while the current one is finishing, so they land during
// the grid barrier.  The stencil operand (the CG vector on the CTA's
// aggregates and their 8 neighbours) is staged in shared memory per phase,
// pre-multiplied by the FP16 block scales and with the sigma_3 sign flips of
// D_c^dag = sigma_3 D_c sigma_3 applied.  In tensor memory (TM = 1, 2) the
// CTA takes all 512 columns of its SM and the operator is written there once
// per launch: TM = 1 keeps it as each thread's share of rows and columns and
// forms the products with packed FP32 FMAs; TM = 2 (FP16 operator) keeps the
// CTA's first 128 rows as the A operand of tcgen05.mma and forms the stencil
// as one MMA tile per phase (see kMmaRows).
//
// Iteration, two forms with the same iterates in exact arithmetic.
// Textbook CGLS (cgls_body: two grid-wide exchanges of partial sums, which
// also serve as the grid barriers):
//   q = D_c p,  alpha = gamma/|q|^2,  y += alpha p,  r -= alpha q,
//   s = D_c^dag r,  gamma' = |s|^2,  beta = gamma'/gamma,  p = s + beta p
// with the vector updates done while staging (p and r double-buffered).
// Chronopoulos-Gear (cgls_body_tag, the default): one exchange per iteration,
// the vectors read across CTAs carrying epoch tags instead of barriers.
#include <atomic>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "mg_launch.h"
#include "mg_ptx.cuh"
#include "mg_sync.cuh"

namespace wmg {

constexpr int kCglsThreads = 512;
constexpr int kXchScratch = kXchMaxNV * (32 + kXchMaxGrid + 1);   // floats for xch_allreduce<3>
constexpr long long kCopyWaitLimit = 4000000LL;   // polls of a bulk-copy mbarrier before giving up

// Four consecutive rows a..a+3 of one column of a unit, as complex FP32 pairs
// (re, im).  FP32: 32 bytes; FP16: 16 bytes (the block scale is carried by
// the staged operand).
template <bool H16> struct UnitOp;
template <> struct UnitOp<false> {
    using type = float2;
    static constexpr int bytes = 8;
    static __device__ __forceinline__ void words(const uint32_t* w, float2 (&v)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = make_float2(__uint_as_float(w[2 * q]), __uint_as_float(w[2 * q + 1]));
    }
    static __device__ __forceinline__ void quad(const float2* p, float2 (&v)[4]) {
        const float4 w0 = reinterpret_cast<const float4*>(p)[0];
        const float4 w1 = reinterpret_cast<const float4*>(p)[1];
        v[0] = make_float2(w0.x, w0.y);
        v[1] = make_float2(w0.z, w0.w);
        v[2] = make_float2(w1.x, w1.y);
        v[3] = make_float2(w1.z, w1.w);
    }
};
template <> struct UnitOp<true> {
    using type = __half2;
    static constexpr int bytes = 4;
    static __device__ __forceinline__ void words(const uint32_t* w, float2 (&v)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __half22float2(*reinterpret_cast<const __half2*>(w + q));
    }
    static __device__ __forceinline__ void quad(const __half2* p, float2 (&v)[4]) {
        const uint4 w = *reinterpret_cast<const uint4*>(p);
        v[0] = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
        v[1] = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
        v[2] = __half22float2(*reinterpret_cast<const __half2*>(&w.z));
        v[3] = __half22float2(*reinterpret_cast<const __half2*>(&w.w));
    }
};

// vectors of one phase (see the staging rules in cgls_phase)
struct CglsPhase {
    const float2* in;      // ST_IN: operand
    const float2* s;       // ST_P: s
    const float2* p_old;   // ST_P: previous direction (ignored when first)
    float2* p_new;         // ST_P: own entries of the new direction; ST_R: current direction (read)
    const float2* r_old;   // ST_R
    const float2* q;       // ST_R
    float2* r_new;         // ST_R
    float2* y;             // ST_R
    float2* out;
    float coef;            // beta (ST_P) or alpha (ST_R)
    bool first;
    // epoch-tagged vectors (two 64-bit words per entry): ST_TAG stages tin at
    // epoch etag; EPI_TAG stores out to tout at epoch etag_out; EPI_CG_TAG (the
    // second stencil of the Chronopoulos-Gear form): out = w = D_c^dag u is not
    // stored; p = s + beta p, z = w + beta z, q = u + beta q, y += alpha p,
    // r -= alpha q, s -= alpha z on the own rows (first: no beta terms), with s
    // and u in the tagged buffers ts, tu (s' stored at epoch etag_out)
    float2 *cp, *cz, *cq, *cy, *cr;
    float alpha, beta;
    const unsigned long long* tin;
    unsigned long long *tout, *ts, *tu;
    unsigned int etag, etag_out;
    int own_out;   // EPI_TAG with own-row vectors in shared memory: the one (OV_S, OV_U) that keeps out
    bool stop;   // set by phase when its pre-emit step declined the epilogue
};
enum { ST_IN = 0, ST_P = 1, ST_R = 2, ST_TAG = 3 };
// pre-emit step of a phase: runs (collectively) between the stencil's products
// and its epilogue; 1 = emit, 0 = stop without emitting, -1 = failure
struct NoPre {
    __device__ int operator()() const { return 1; }
};
enum { EPI_STORE = 0, EPI_TAG = 1, EPI_CG_TAG = 2 };
enum { OV_P = 0, OV_Z = 1, OV_Q = 2, OV_Y = 3, OV_R = 4, OV_S = 5, OV_U = 6, OV_COUNT = 7 };

constexpr int kStageRegs = 4;   // staged operand entries per thread kept as precomputed offsets

// Tensor-core products (TM == 2, FP16 operator): the first kMmaRows rows of a
// CTA are one MMA tile, row r in TMEM lane r, column k holding the FP16 complex
// entry k = d nc + b (low half Re, high half Im: the K-major A operand with
// K = 2 * 9nc real elements).  B (kMmaN x 2K, K-major core matrices in shared
// memory) holds per aggregate xl of the CTA four rows: the staged operand x as
// FP16 hi + lo parts (x = hi + lo to ~22 bits, after a per-aggregate power-of-
// two scale), laid out so that row 4xl (Re) pairs (Re a, Im a) with (Re x, -Im x)
// and row 4xl+1 (Im) with (Im x, Re x); rows 4xl+2, 4xl+3 the same for lo.  So
// D[r][4xl + {0,1,2,3}] summed in pairs is Re, Im of (D_c x)_r.  Rows beyond the
// tile (at most kMmaRemWarps) are summed on the CUDA cores, one warp each.
constexpr int kMmaRows = 128;
constexpr int kMmaN = 32;
constexpr int kMmaAgg = kMmaN / 4;
constexpr int kMmaRemWarps = kCglsThreads / 32 - 4;
// B tile: core matrices adjacent in N 128 bytes apart, adjacent in K one
// group of kMmaN / 8 core matrices plus 16 bytes apart (so that the 16-byte
// stores of 8 consecutive K groups by 8 lanes hit distinct banks)
constexpr int kMmaLbo = (kMmaN / 8) * 128 + 16;
constexpr int kMmaMaxAcc = 4;   // accumulators the K steps alternate over (TMEM columns permitting)
// the per-accumulator row partials of the epilogue live in the reduction buffer
static_assert(kMmaMaxAcc * kMmaRows * 16 <= 4 * kCglsThreads * 8, "reduction buffer too small for the partials");
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
// exponent es with max * 2^es in [2^13, 2^14), max given by its float bits (>= 0)
__device__ __forceinline__ int agg_exp(int bits) {
    if (bits <= 0) return 0;
    const int es = 13 - (((bits >> 23) & 0xff) - 127);
    return min(max(es, -126), 126);
}
// One chain of MMAs (K = 16 each) of a tile product: n steps, the first at A
// column `at` and B descriptor `bd`, the next ones astep columns and bstep
// descriptor units (16 bytes; the shared-memory window keeps the address field
// below 2^14) further, all accumulating into d.  The issuing thread's loop is
// the critical path, so it only adds constants.
__device__ __forceinline__ void issue_chain(uint32_t d, uint32_t at, uint64_t bd, int n, uint32_t astep,
                                            uint64_t bstep) {
    constexpr uint32_t idesc = idesc_f16(kMmaRows, kMmaN);
    mma_f16_ts(d, at, bd, idesc, 0u);
#pragma unroll 4
    for (int i = 1; i < n; ++i) {
        at += astep;
        bd += bstep;
        mma_f16_ts(d, at, bd, idesc, 1u);
    }
}
__device__ __forceinline__ uint32_t half_pair(__half lo, __half hi) {
    __half2 h = __halves2half2(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <bool H16, int TM> struct CglsCta {
    using OT = typename UnitOp<H16>::type;
    // words of one row quad of one column: FP16 4 x half2, FP32 4 x float2
    static constexpr int kWpq = H16 ? 4 : 8;
    static constexpr int kQpc = 32 / kWpq;   // quads per 32-column TMEM chunk
    const CglsArgs& a;
    int nc, K, nvh, RU, H, u0, u1, nu, X0, nX;
    int W, NG, NW;
    bool resident;
    uint64_t* mbar;
    cx<float>* red;
    cx<float>* xs;
    unsigned char* slots;
    // own-row vectors of the tagged form in shared memory (nullptr: in global
    // memory): [OV_* 7][own row], own row = the index of the row among the CTA's
    cx<float>* ov = nullptr;
    int ov_n = 0;
    int buf = 0;
    long long gw_next = 0;     // next wave to consume (all threads)
    long long gw_issued = 0;   // next wave to copy (thread 0)
    bool loaded = false;       // resident copy issued
    // staging entries of this thread (when nX * K <= kStageRegs * blockDim.x):
    // global offset Y*nc + b, FP16 block scale, flags (1: own entry, 2: b >= nc/2,
    // bits 2..: the entry's aggregate among the CTA's)
    bool pre = false;
    // TMEM-resident operator (TM): this thread's quad qd and column split ks
    // (k = ks, ks + KS, ...), its TMEM lane/column base and the CTA-wide chunk count
    int q_ks = 0, q_qd = 0, q_KS = 1, q_quads = 0, q_nch = 0;
    bool q_act = false;
    uint32_t q_taddr = 0, tm_base = 0;
    int st_o[kStageRegs];
    float st_s[kStageRegs];
    int st_f[kStageRegs];
    bool sfail = false;   // a tagged staging wait gave up (error flag raised)
    // tensor-core products (TM == 2): B tile, rows beyond the MMA tile, the
    // per-aggregate maxima of the staged operand ([2][kMmaAgg] float bits,
    // alternating between phases), commits issued, a commit not seen complete
    unsigned char* bt = nullptr;
    uint32_t* rop = nullptr;
    int* amax = nullptr;
    int mph = 0;
    uint32_t mma_n = 0;
    bool mma_out = false;
    int rows_m = 0, rem = 0, nacc = 1;
    uint32_t dcol = 0;
    // per-thread row constants (TM == 2): the row this thread emits (-1: none),
    // its output offset X nc + row, sign rule and aggregate; the aggregate of
    // the row whose accumulator columns it reads (-1: none)
    int e_row = -1, e_o = 0, e_xl = 0, p_xl = -1;
    bool e_neg = false;

    __device__ CglsCta(const CglsArgs& args, unsigned char* sm) : a(args) {
        nc = a.nc; K = 9 * nc; nvh = nc >> 1; RU = a.sh.ru; H = nc / RU;
        const long long NU = (long long)a.g.Vc * H, G = gridDim.x;
        u0 = (int)(blockIdx.x * NU / G);
        u1 = (int)((blockIdx.x + 1) * NU / G);
        nu = u1 - u0;
        X0 = u0 / H;
        nX = (u1 - 1) / H - X0 + 1;
        resident = a.sh.resident != 0;
        NG = resident ? 1 : a.sh.groups;
        W = resident ? nu : a.sh.wave;
        NW = (nu + W - 1) / W;
        mbar = reinterpret_cast<uint64_t*>(sm);
        red = reinterpret_cast<cx<float>*>(sm + 256);
        xs = red + (resident ? 1 : 2) * a.sh.red_n;
        slots = sm + a.sh.slot_off;
        if (a.sh.own_off > 0 && (a.form == CGLS_CG_TAGGED || a.form == CGLS_PROBE_STENCILS)) {
            ov = reinterpret_cast<cx<float>*>(sm + a.sh.own_off);
            ov_n = a.sh.nu_max * RU;
        }
        if (TM == 2) {
            bt = sm + a.sh.bt_off;
            rop = reinterpret_cast<uint32_t*>(sm + a.sh.rop_off);
            amax = reinterpret_cast<int*>(sm + 64);
            rows_m = min(nu * RU, kMmaRows);
            rem = nu * RU - rows_m;
            dcol = (uint32_t)(32 * ((K + 31) / 32));
            nacc = a.sh.mma_acc;
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            if (warp < 4 && (int)threadIdx.x < rows_m)
                e_row = threadIdx.x;
            else if (warp >= 4 && warp - 4 < rem)
                e_row = kMmaRows + warp - 4;   // whole warp sums it; lane 0 emits
            if (e_row >= 0) {
                const int jj = e_row / RU, ain = e_row - jj * RU, u = u0 + jj, X = u / H, row = (u - X * H) * RU + ain;
                e_o = X * nc + row;
                e_neg = row >= nvh;
                e_xl = X - X0;
            }
            const int rq = 32 * (warp & 3) + lane;
            if (rq < rows_m) p_xl = (u0 + rq / RU) / H - X0;
        }
        pre = nX * K <= kStageRegs * (int)blockDim.x;
        if (pre) {
#pragma unroll
            for (int q = 0; q < kStageRegs; ++q) {
                const int i = threadIdx.x + q * blockDim.x;
                st_o[q] = -1;
                st_s[q] = 1.f;
                st_f[q] = 0;
                if (i < nX * K) {
                    const int xl = i / K, kk = i - xl * K, d = kk / nc, b = kk - d * nc, X = X0 + xl;
                    st_o[q] = __ldg(a.nbr + (size_t)X * 9 + d) * nc + b;
                    if (H16) st_s[q] = __ldg(a.su + (size_t)X * 9 + d);
                    st_f[q] = ((d == 0 && owned(X, b)) ? 1 : 0) | (b >= nvh ? 2 : 0) | (xl << 2);
                }
            }
        }
    }
    __device__ bool owned(int X, int b) const {
        long long u = (long long)X * H + b / RU;
        return u >= u0 && u < u1;
    }
    __device__ size_t unit_bytes() const { return (size_t)K * RU * UnitOp<H16>::bytes; }
    // thread 0: copy the units of wave gw into its slot group
    __device__ void issue(long long gw) {
        const int grp = resident ? 0 : (int)(gw % NG);
        const int iw = resident ? 0 : (int)(gw % NW);
        const int j0 = iw * W, n = min(W, nu - j0);
        const uint32_t ub = (uint32_t)unit_bytes();
        mbar_expect_tx(mbar + grp, ub * (uint32_t)n);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(a.Au) + (size_t)(u0 + j0) * ub;
        for (int j = 0; j < n; ++j)
            bulk_copy_g2s(slots + (size_t)(grp * W + j) * a.sh.stride, src + (size_t)j * ub, ub, mbar + grp);
    }
    __device__ void start() {
        if (TM) {
            start_tmem();
            return;
        }
        if (threadIdx.x == 0) {
            for (int i = 0; i < NG; ++i) mbar_init(mbar + i, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (resident) {
                issue(0);
            } else {
                for (int i = 0; i < NG; ++i) issue(i);
            }
        }
        gw_issued = resident ? 1 : NG;
        loaded = true;
    }
    // TM: allocate all 512 TMEM columns (one CTA per SM) and copy this thread's
    // share of the operator into its lane: thread (warp w, lane l) owns lane
    // 32 (w % 4) + l, columns 128 (w / 4) .. +127
    __device__ void start_tmem() {
        __shared__ uint32_t s_taddr;
        const int warp = threadIdx.x >> 5, T = blockDim.x;
        if (warp == 0) {
            tmem_alloc(&s_taddr, 512);
            tmem_relinquish();
        }
        if (TM == 2) {
            if (threadIdx.x == 0) {
                mbar_init(mbar, nacc);   // MMA completion: one commit per issuing thread
                fence_mbar_init();
            }
            if (threadIdx.x < 2 * kMmaAgg) amax[threadIdx.x] = 0;
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const uint32_t base = s_taddr;
        tm_base = base;
        if constexpr (TM == 2) {
            // row r of the CTA in lane r (warps w and w + 4k share lanes 32 (w % 4)..,
            // and split the 32-column chunks); zeros past K and in lanes >= rows_m
            const int lane = threadIdx.x & 31, r = 32 * (warp & 3) + lane;
            const uint32_t* src = nullptr;
            if (r < rows_m) {
                const int j = r / RU, ain = r - j * RU;
                src = reinterpret_cast<const uint32_t*>(reinterpret_cast<const unsigned char*>(a.Au) +
                                                        (size_t)(u0 + j) * unit_bytes()) + ain;
            }
            const int nch = (K + 31) / 32;
            for (int c = warp >> 2; c < nch; c += T / 128) {
                uint32_t w[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int k = 32 * c + i;
                    w[i] = (src && k < K) ? __ldg(src + (size_t)k * RU) : 0u;
                }
                tmem_st32(base + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * c, w);
            }
            // rows beyond the MMA tile: rop[rr][k] in shared memory
            for (int i = threadIdx.x; i < rem * K; i += T) {
                const int rr = i / K, k = i - rr * K, r2 = kMmaRows + rr, j = r2 / RU, ain = r2 - j * RU;
                rop[i] = __ldg(reinterpret_cast<const uint32_t*>(reinterpret_cast<const unsigned char*>(a.Au) +
                                                                 (size_t)(u0 + j) * unit_bytes()) +
                               (size_t)k * RU + ain);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            loaded = true;
            return;
        }
        q_quads = (nu * RU) >> 2;
        q_KS = max(1, T / q_quads);
        q_act = (int)threadIdx.x < q_quads * q_KS;
        q_ks = threadIdx.x / q_quads;
        q_qd = threadIdx.x - q_ks * q_quads;
        q_nch = ((K + q_KS - 1) / q_KS + kQpc - 1) / kQpc;   // chunks of the thread with ks = 0
        q_taddr = base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(128 * (warp >> 2));
        const int r = 4 * q_qd, j = r / RU, ain = r - j * RU;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(
            reinterpret_cast<const unsigned char*>(a.Au) + (size_t)(u0 + j) * unit_bytes()) + (size_t)ain * (kWpq / 4);
        for (int c = 0; c < q_nch; ++c) {
            uint32_t w[32];
#pragma unroll
            for (int i = 0; i < kQpc; ++i) {
                const int k = q_ks + (c * kQpc + i) * q_KS;
                const bool ok = q_act && k < K;
#pragma unroll
                for (int v = 0; v < kWpq; ++v) w[i * kWpq + v] = ok ? __ldg(src + (size_t)k * RU * (kWpq / 4) + v) : 0u;
            }
            tmem_st32(q_taddr + 32 * c, w);
        }
        tmem_wait_st();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        loaded = true;
    }
    // thread 0: wait for every copy still in flight (before the CTA may exit);
    // TM: release the tensor memory
    __device__ void drain() {
        if (TM) {
            // a commit whose completion a phase gave up on: wait (bounded) once more
            // before the columns are released
            if (TM == 2 && mma_out && threadIdx.x == 0) mbar_wait(mbar, (mma_n - 1) & 1u, kCopyWaitLimit);
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if ((threadIdx.x >> 5) == 0) tmem_dealloc(tm_base, 512);
            return;
        }
        if (threadIdx.x != 0 || !loaded) return;
        if (resident) {
            mbar_wait(mbar, 0, kCopyWaitLimit);
        } else {
            for (long long g = gw_next; g < gw_issued; ++g) mbar_wait(mbar + g % NG, (uint32_t)((g / NG) & 1), kCopyWaitLimit);
        }
    }

    // operand entry at global offset o, formed per STAGE (see phase); own: this
    // CTA owns the entry and performs its vector updates
    template <int STAGE> __device__ __forceinline__ cx<float> form(const CglsPhase& ph, int o, bool own, float& n1) {
        cx<float> v;
        if (STAGE == ST_IN) {
            v = ld<float>(ph.in + o);
        } else if (STAGE == ST_TAG) {
            float2 t;
            if (!tag_wait(ph.tin + 2 * (size_t)o, ph.etag, a.err, t)) sfail = true;
            v = cx<float>(t.x, t.y);
        } else if (STAGE == ST_P) {
            v = ld<float>(ph.s + o);
            if (!ph.first) v = v + ph.coef * ld<float>(ph.p_old + o);
            if (own) st<float>(ph.p_new + o, v);
        } else {
            v = ld<float>(ph.r_old + o) - ph.coef * ld<float>(ph.q + o);
            if (own) {
                st<float>(ph.r_new + o, v);
                st<float>(ph.y + o, ld<float>(ph.y + o) + ph.coef * ld<float>(ph.p_new + o));
                n1 += norm2(v);
            }
        }
        return v;
    }

    // output row o = X * nc + row of the stencil (own row j of the CTA): EPI_STORE /
    // EPI_TAG store it (n0 += |out|^2); EPI_CG_TAG applies the updates
    // (n0 += |s'|^2, n1 += |r'|^2), on the own-row vectors in shared memory when
    // the shape has room for them
    template <int EPI> __device__ __forceinline__ void emit(const CglsPhase& ph, size_t o, int j, cx<float> w, float& n0,
                                                            float& n1) {
        if (EPI == EPI_STORE) {
            st<float>(ph.out + o, w);
            n0 += norm2(w);
        } else if (EPI == EPI_TAG) {
            tag_store(ph.tout + 2 * o, w.r, w.i, ph.etag_out);
            if (ov) ov[ph.own_out * ov_n + j] = w;
            n0 += norm2(w);
        } else if (EPI == EPI_CG_TAG) {
            cx<float> s, u, p0, z0, q0, y0, r0;
            if (ov) {
                s = ov[OV_S * ov_n + j];
                u = ov[OV_U * ov_n + j];
                y0 = ov[OV_Y * ov_n + j];
                r0 = ov[OV_R * ov_n + j];
                if (!ph.first) {
                    p0 = ov[OV_P * ov_n + j];
                    z0 = ov[OV_Z * ov_n + j];
                    q0 = ov[OV_Q * ov_n + j];
                }
            } else {
                float2 s2, u2;
                tag_load(ph.ts + 2 * o, 0u, s2);   // own entries, written by this CTA
                tag_load(ph.tu + 2 * o, 0u, u2);
                s = cx<float>(s2.x, s2.y);
                u = cx<float>(u2.x, u2.y);
                y0 = ld<float>(ph.cy + o);
                r0 = ld<float>(ph.cr + o);
                if (!ph.first) {
                    p0 = ld<float>(ph.cp + o);
                    z0 = ld<float>(ph.cz + o);
                    q0 = ld<float>(ph.cq + o);
                }
            }
            cx<float> p = s, z = w, q = u;
            if (!ph.first) {
                p = p + ph.beta * p0;
                z = z + ph.beta * z0;
                q = q + ph.beta * q0;
            }
            const cx<float> sn = s - ph.alpha * z, rn = r0 - ph.alpha * q, yn = y0 + ph.alpha * p;
            if (ov) {
                ov[OV_P * ov_n + j] = p;
                ov[OV_Z * ov_n + j] = z;
                ov[OV_Q * ov_n + j] = q;
                ov[OV_Y * ov_n + j] = yn;
                ov[OV_R * ov_n + j] = rn;
                ov[OV_S * ov_n + j] = sn;
            } else {
                st<float>(ph.cp + o, p);
                st<float>(ph.cz + o, z);
                st<float>(ph.cq + o, q);
                st<float>(ph.cy + o, yn);
                st<float>(ph.cr + o, rn);
            }
            tag_store(ph.ts + 2 * o, sn.r, sn.i, ph.etag_out);
            n0 += norm2(sn);
            n1 += norm2(rn);
        }
    }

    // TM == 2 staging: the thread's entries (the coalesced mapping of the other
    // shapes) signed and block-scaled into xs, each aggregate's maximum |x|
    // through a warp reduction and one shared atomic per aggregate and warp;
    // after a barrier thread t forms B from entries 4t..4t+3 (one aggregate xl,
    // one 8-element K group): x * 2^es split into FP16 hi + lo in its 16-byte
    // slots of the four B rows of xl.  Collective; ends with the async-proxy
    // fence (the caller's barrier then orders the tile before the MMAs).
    template <bool DAG> __device__ __forceinline__ void stage_mma(const cx<float> (&v)[kStageRegs]) {
        const int T = blockDim.x;
        int* am = amax + kMmaAgg * mph;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int q = 0; q < kStageRegs; ++q) {
            int xl = -1;
            int bits = 0;
            if (st_o[q] >= 0) {
                cx<float> w = v[q];
                if (DAG && (st_f[q] & 2)) w = cx<float>(-w.r, -w.i);
                if (H16) w = st_s[q] * w;
                xs[threadIdx.x + q * T] = w;
                xl = st_f[q] >> 2;
                bits = __float_as_int(fmaxf(fabsf(w.r), fabsf(w.i)));
            }
            // the warp's 32 consecutive entries span at most two aggregates (K >= 32;
            // inactive entries, xl = -1, only at the end): one reduction each
            const int x0 = __shfl_sync(0xffffffffu, xl, 0), x1 = __shfl_sync(0xffffffffu, xl, 31);
            const int m0 = __reduce_max_sync(0xffffffffu, xl == x0 ? bits : 0);
            if (lane == 0 && x0 >= 0) atomicMax(am + x0, m0);
            if (x1 != x0) {
                const int m1 = __reduce_max_sync(0xffffffffu, xl == x0 ? 0 : bits);
                if (lane == 31 && x1 >= 0) atomicMax(am + x1, m1);
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < kMmaAgg) amax[kMmaAgg * (mph ^ 1) + threadIdx.x] = 0;   // next phase's maxima
        const int i0 = kStageRegs * (int)threadIdx.x;
        if (i0 < nX * K) {
            const int xl = i0 / K;
            const float sc = pow2f(agg_exp(am[xl]));
            const float4* x4 = reinterpret_cast<const float4*>(xs + i0);
            const float4 xa = x4[0], xb = x4[1];
            const float re[4] = {xa.x * sc, xa.z * sc, xb.x * sc, xb.z * sc};
            const float im[4] = {xa.y * sc, xa.w * sc, xb.y * sc, xb.w * sc};
            uint32_t rh[kStageRegs], ih[kStageRegs], rl[kStageRegs], il[kStageRegs];
#pragma unroll
            for (int q = 0; q < kStageRegs; ++q) {
                const __half reh = __float2half_rn(re[q]), imh = __float2half_rn(im[q]);
                const __half rel = __float2half_rn(re[q] - __half2float(reh));
                const __half iml = __float2half_rn(im[q] - __half2float(imh));
                rh[q] = half_pair(reh, __hneg(imh));
                ih[q] = half_pair(imh, reh);
                rl[q] = half_pair(rel, __hneg(iml));
                il[q] = half_pair(iml, rel);
            }
            unsigned char* dst = bt + (size_t)((i0 - xl * K) >> 2) * kMmaLbo + 64 * xl;
            *reinterpret_cast<uint4*>(dst) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
            *reinterpret_cast<uint4*>(dst + 16) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
            *reinterpret_cast<uint4*>(dst + 32) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
            *reinterpret_cast<uint4*>(dst + 48) = make_uint4(il[0], il[1], il[2], il[3]);
        }
        fence_proxy_async();
        mph ^= 1;
    }

    // TM == 2 products and epilogue (after the staging barrier): lane 0 of warps
    // 0 .. nacc-1 issue the 9nc/8 MMAs of the tile as nacc chains into nacc
    // accumulators and commit them to the mbarrier; meanwhile warps 4.. sum the
    // rows beyond the tile; every thread waits for the commits; warp 4j + q
    // reads accumulator j on lane quadrant q and keeps its row's four columns
    // in part[j][row]; pre_emit; one emitting thread per row sums the partials.
    template <bool DAG, int EPI, typename Pre>
    __device__ bool mma_phase(CglsPhase& ph, float& n0, float& n1, Pre& pre_emit) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0 && warp < nacc) {
            // K steps k8 = warp, warp + nacc, ... into accumulator `warp`: nacc
            // independent chains issued by nacc threads, each committing once
            constexpr uint64_t kStep = (2 * kMmaLbo) >> 4;
            tc_fence_after();
            const uint64_t bd = smem_desc(smem_u32(bt), kMmaLbo, 128) + kStep * (uint64_t)warp;
            issue_chain(tm_base + dcol + kMmaN * warp, tm_base + 8 * warp, bd, (K / 8 - warp + nacc - 1) / nacc,
                        8u * nacc, kStep * (uint64_t)nacc);
            mma_commit(mbar);
        }
        const int* am = amax + kMmaAgg * (mph ^ 1);   // this phase's maxima
        cx<float> ysum(0.f, 0.f);
        if (warp >= 4 && e_row >= 0) {
            const float2* xv = reinterpret_cast<const float2*>(xs) + (size_t)e_xl * K;
            const __half2* ar = reinterpret_cast<const __half2*>(rop) + (size_t)(warp - 4) * K;
            float yr = 0.f, yi = 0.f;
            for (int k = lane; k < K; k += 32) {
                const float2 av = __half22float2(ar[k]), x = xv[k];
                yr = fmaf(av.x, x.x, fmaf(-av.y, x.y, yr));
                yi = fmaf(av.x, x.y, fmaf(av.y, x.x, yi));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                yr += __shfl_xor_sync(0xffffffffu, yr, o);
                yi += __shfl_xor_sync(0xffffffffu, yi, o);
            }
            ysum = cx<float>(yr, yi);
        }
        const bool got = mbar_wait(mbar, mma_n & 1u, kCopyWaitLimit);
        ++mma_n;
        tc_fence_after();
        // accumulator j of lane quadrant w % 4 read by warp w = 4 j + quadrant (the
        // four warps of a quadrant load in parallel); its row's four columns
        // into part[j][row] (the reduction buffer, unused by this path)
        float4* part = reinterpret_cast<float4*>(red);
        if ((warp >> 2) < nacc) {
            const int rq = 32 * (warp & 3) + lane;
            uint32_t d[32];
            tmem_ld32(tm_base + ((uint32_t)(32 * (warp & 3)) << 16) + dcol + kMmaN * (warp >> 2), d);
            if (p_xl >= 0) {
                // columns 4 p_xl .. 4 p_xl + 3 by a select tree on the bits of p_xl
                // (constant register indices only)
                uint32_t h[16], g[8], f[4];
#pragma unroll
                for (int i = 0; i < 16; ++i) h[i] = (p_xl & 4) ? d[16 + i] : d[i];
#pragma unroll
                for (int i = 0; i < 8; ++i) g[i] = (p_xl & 2) ? h[8 + i] : h[i];
#pragma unroll
                for (int i = 0; i < 4; ++i) f[i] = (p_xl & 1) ? g[4 + i] : g[i];
                part[(warp >> 2) * kMmaRows + rq] = make_float4(__uint_as_float(f[0]), __uint_as_float(f[1]),
                                                                __uint_as_float(f[2]), __uint_as_float(f[3]));
            }
        }
        tc_fence_before();
        const int r = threadIdx.x;
        if (__syncthreads_or(!got)) {
            if (threadIdx.x == 0) atomicExch(a.err, 3);
            mma_out = true;
            return false;
        }
        const int go = pre_emit();
        if (go < 0) return false;
        if (go == 0) {
            ph.stop = true;
            return true;
        }
        if (e_row >= 0 && (warp < 4 || lane == 0)) {
            cx<float> sum = ysum;
            if (warp < 4) {
                float4 c = part[r];
                for (int j = 1; j < nacc; ++j) {
                    const float4 e = part[j * kMmaRows + r];
                    c.x += e.x; c.y += e.y; c.z += e.z; c.w += e.w;
                }
                const float inv = pow2f(-agg_exp(am[e_xl]));
                sum = cx<float>((c.x + c.z) * inv, (c.y + c.w) * inv);
            }
            if (DAG && e_neg) sum = cx<float>(-sum.r, -sum.i);
            emit<EPI>(ph, (size_t)e_o, e_row, sum, n0, n1);
        }
        return true;
    }

    // One stencil application out = D_c (or D_c^dag) x on the CTA's rows, the
    // operand x formed while staging:
    //   ST_IN: x = in
    //   ST_P : x = s + beta p_old (first: s); own entries -> p_new
    //   ST_R : x = r_old - alpha q; own entries -> r_new, y += alpha p_new, n1 += |x|^2
    // n0 accumulates |out|^2 over the CTA's rows.  pre_emit() runs after the
    // products and before the first output row is emitted (see NoPre); false
    // on a failed wait.
    template <int STAGE, bool DAG, int EPI = EPI_STORE, typename Pre = NoPre>
    __device__ bool phase(CglsPhase& ph, float& n0, float& n1, Pre&& pre_emit = Pre()) {
        ph.stop = false;
        const int T = blockDim.x;
        if (pre) {
            cx<float> v[kStageRegs];
            if (STAGE == ST_TAG) {
                // all loads first, then re-poll only the entries not yet at epoch etag
                unsigned int okm = 0;
#pragma unroll
                for (int q = 0; q < kStageRegs; ++q) {
                    float2 t = make_float2(0.f, 0.f);
                    if (st_o[q] < 0 || tag_load(ph.tin + 2 * (size_t)st_o[q], ph.etag, t)) okm |= 1u << q;
                    v[q] = cx<float>(t.x, t.y);
                }
                long long spins = 0;
                while (okm != (1u << kStageRegs) - 1u) {
#pragma unroll
                    for (int q = 0; q < kStageRegs; ++q)
                        if (!((okm >> q) & 1u)) {
                            float2 t;
                            if (tag_load(ph.tin + 2 * (size_t)st_o[q], ph.etag, t)) {
                                okm |= 1u << q;
                                v[q] = cx<float>(t.x, t.y);
                            }
                        }
                    if (okm == (1u << kStageRegs) - 1u) break;
                    if (*(volatile int*)a.err) { sfail = true; break; }
                    if (++spins > kExchangeSpinLimit) { atomicExch(a.err, 1); sfail = true; break; }
                    if (spins > 32) __nanosleep(20);
                }
            } else {
#pragma unroll
                for (int q = 0; q < kStageRegs; ++q)
                    if (st_o[q] >= 0) v[q] = form<STAGE>(ph, st_o[q], (st_f[q] & 1) != 0, n1);
            }
            if constexpr (TM == 2) {
                stage_mma<DAG>(v);
            } else {
#pragma unroll
                for (int q = 0; q < kStageRegs; ++q)
                    if (st_o[q] >= 0) {
                        cx<float> w = v[q];
                        if (DAG && (st_f[q] & 2)) w = cx<float>(-w.r, -w.i);
                        if (H16) w = st_s[q] * w;
                        xs[threadIdx.x + q * T] = w;
                    }
            }
        } else {
            for (int i = threadIdx.x; i < nX * K; i += T) {
                const int xl = i / K, kk = i - xl * K, d = kk / nc, b = kk - d * nc;
                const int X = X0 + xl;
                const int o = __ldg(a.nbr + (size_t)X * 9 + d) * nc + b;
                cx<float> w = form<STAGE>(ph, o, d == 0 && owned(X, b), n1);
                if (DAG && b >= nvh) w = cx<float>(-w.r, -w.i);
                if (H16) w = __ldg(a.su + (size_t)X * 9 + d) * w;
                xs[i] = w;
            }
        }
        if (__syncthreads_or(sfail)) return false;
        if constexpr (TM == 2) return mma_phase<DAG, EPI>(ph, n0, n1, pre_emit);
        const float2* xs2 = reinterpret_cast<const float2*>(xs);
        if constexpr (TM != 0) {
            const int rows = nu * RU;
            const int r = 4 * q_qd, j = r / RU;
            const float2* xv = xs2 + (size_t)((u0 + j) / H - X0) * K;
            float2 P[4], Q[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { P[q] = make_float2(0.f, 0.f); Q[q] = make_float2(0.f, 0.f); }
            for (int c = 0; c < q_nch; ++c) {
                uint32_t w[32];
                tmem_ld32(q_taddr + 32 * c, w);
                if (q_act) {
#pragma unroll
                    for (int i = 0; i < kQpc; ++i) {
                        const int k = q_ks + (c * kQpc + i) * q_KS;
                        if (k < K) {
                            const float2 x = xv[k];
                            const float2 xw = make_float2(x.y, x.x);
                            float2 av[4];
                            UnitOp<H16>::words(w + i * kWpq, av);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                P[q] = __ffma2_rn(av[q], x, P[q]);
                                Q[q] = __ffma2_rn(av[q], xw, Q[q]);
                            }
                        }
                    }
                }
            }
            if (q_act)
#pragma unroll
                for (int q = 0; q < 4; ++q) red[q_ks * rows + r + q] = cx<float>(P[q].x - P[q].y, Q[q].x + Q[q].y);
            __syncthreads();
            const int go = pre_emit();
            if (go < 0) return false;
            if (go == 0) {
                ph.stop = true;
                return true;
            }
            for (int rr = threadIdx.x; rr < rows; rr += T) {
                cx<float> sum = red[rr];
                for (int ks = 1; ks < q_KS; ++ks) sum = sum + red[ks * rows + rr];
                const int jj = rr / RU, ain = rr - jj * RU, u = u0 + jj, X = u / H, row = (u - X * H) * RU + ain;
                if (DAG && row >= nvh) sum = cx<float>(-sum.r, -sum.i);
                emit<EPI>(ph, (size_t)X * nc + row, rr, sum, n0, n1);
            }
            return true;
        } else {
        for (int iw = 0; iw < NW; ++iw) {
            const int j0 = iw * W, n = min(W, nu - j0), rows = n * RU, quads = rows >> 2;
            const int grp = resident ? 0 : (int)(gw_next % NG);
            const uint32_t par = resident ? 0u : (uint32_t)((gw_next / NG) & 1);
            if (!mbar_wait(mbar + grp, par, kCopyWaitLimit)) atomicExch(a.err, 2);
            const unsigned char* base = slots + (size_t)(resident ? j0 : grp * W) * a.sh.stride;
            const int KS = max(1, T / quads);
            cx<float>* rb = red + buf * a.sh.red_n;
            for (int t = threadIdx.x; t < quads * KS; t += T) {
                const int ks = t / quads, qd = t - ks * quads;
                const int r = 4 * qd, j = r / RU, ain = r - j * RU;
                const int xl = (u0 + j0 + j) / H - X0;
                const OT* A = reinterpret_cast<const OT*>(base + (size_t)j * a.sh.stride) + ain;
                const float2* xv = xs2 + (size_t)xl * K;
                // P_r = sum (Re a x_r, Im a x_i), Q_r = sum (Re a x_i, Im a x_r):
                // Re y_r = P.x - P.y, Im y_r = Q.x + Q.y (packed FP32 FMA)
                float2 P[4], Q[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { P[q] = make_float2(0.f, 0.f); Q[q] = make_float2(0.f, 0.f); }
#pragma unroll 2
                for (int k = ks; k < K; k += KS) {
                    const float2 x = xv[k];
                    const float2 xw = make_float2(x.y, x.x);
                    float2 av[4];
                    UnitOp<H16>::quad(A + (size_t)k * RU, av);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        P[q] = __ffma2_rn(av[q], x, P[q]);
                        Q[q] = __ffma2_rn(av[q], xw, Q[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) rb[ks * rows + r + q] = cx<float>(P[q].x - P[q].y, Q[q].x + Q[q].y);
            }
            __syncthreads();
            if (!resident) {
                ++gw_next;
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    issue(gw_issued);
                    ++gw_issued;
                }
            }
            if (iw == 0) {
                const int go = pre_emit();
                if (go < 0) return false;
                if (go == 0) {
                    ph.stop = true;
                    return true;
                }
            }
            for (int r = threadIdx.x; r < rows; r += T) {
                cx<float> sum = rb[r];
                for (int ks = 1; ks < KS; ++ks) sum = sum + rb[ks * rows + r];
                const int j = r / RU, ain = r - j * RU, u = u0 + j0 + j, X = u / H, row = (u - X * H) * RU + ain;
                if (DAG && row >= nvh) sum = cx<float>(-sum.r, -sum.i);
                emit<EPI>(ph, (size_t)X * nc + row, j0 * RU + r, sum, n0, n1);
            }
            if (!resident) buf ^= 1;
        }
        return true;
        }
    }
};

template <bool H16, int TM> __device__ void cgls_body(const CglsArgs& a, CglsCta<H16, TM>& c) {
    unsigned int e = a.epoch0;   // one epoch per exchange
    // exchange scratch: its own kXchScratch floats after the staging buffer
    float* shr = reinterpret_cast<float*>(c.xs + (size_t)a.sh.nx_max * c.K);
    float2* rbuf[2] = {a.r, a.r1};
    float2* pbuf[2] = {a.p, a.p1};
    // y = 0, r = rc on the own rows; |rc|^2
    float one[1] = {0.f};
    for (int i = threadIdx.x; i < c.nu * c.RU; i += blockDim.x) {
        const int j = i / c.RU, ain = i - j * c.RU, u = c.u0 + j, X = u / c.H;
        const size_t o = (size_t)X * c.nc + (u - X * c.H) * c.RU + ain;
        const float2 v = a.rc[o];
        a.r[o] = v;
        a.y[o] = make_float2(0.f, 0.f);
        one[0] += v.x * v.x + v.y * v.y;
    }
    if (!xch_allreduce<1>(one, a.xch, e++, a.err, shr)) return;
    const float rc2 = one[0];
    int it = 0;
    float r2 = rc2;
    if (rc2 > 0.f && a.maxit > 0) {
        CglsPhase ph{};
        float n0 = 0.f, n1 = 0.f;
        // s = D_c^dag r, gamma = |s|^2
        ph.in = a.r;
        ph.out = a.s;
        c.template phase<ST_IN, true>(ph, n0, n1);
        one[0] = n0;
        if (!xch_allreduce<1>(one, a.xch, e++, a.err, shr)) return;
        float gamma = one[0];
        float beta = 0.f;
        for (;;) {
            const int b = it & 1;
            ph = CglsPhase{};
            ph.s = a.s; ph.p_old = pbuf[b ^ 1]; ph.p_new = pbuf[b]; ph.out = a.q;
            ph.coef = beta; ph.first = (it == 0);
            n0 = 0.f; n1 = 0.f;
            c.template phase<ST_P, false>(ph, n0, n1);
            one[0] = n0;
            if (!xch_allreduce<1>(one, a.xch, e++, a.err, shr)) return;
            const float qq = one[0];
            if (!(qq > 0.f)) break;
            const float alpha = gamma / qq;
            ph = CglsPhase{};
            ph.r_old = rbuf[b]; ph.q = a.q; ph.r_new = rbuf[b ^ 1]; ph.y = a.y; ph.p_new = pbuf[b];
            ph.out = a.s; ph.coef = alpha;
            n0 = 0.f; n1 = 0.f;
            c.template phase<ST_R, true>(ph, n0, n1);
            float two[2] = {n0, n1};
            if (!xch_allreduce<2>(two, a.xch, e++, a.err, shr)) return;
            const float gnew = two[0];
            r2 = two[1];
            ++it;
            if (r2 <= a.tol2 * rc2 || it >= a.maxit) break;
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

// The same CG on D_c^dag D_c in the Chronopoulos-Gear arrangement (same
// iterates in exact arithmetic): with u = D_c s and w = D_c^dag u = D_c^dag D_c s,
// both scalars of an iteration come from the first stencil,
//   gamma = |s|^2,  delta = <w, s> = |u|^2,  beta = gamma/gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old)   (first: gamma/delta),
// and the recurrences p = s + beta p, z = w + beta z (= D^dag D p),
// q = u + beta q (= D p), y += alpha p, r -= alpha q, s -= alpha z follow the
// second.  Per iteration: u = D_c s; one exchange of (|u|^2, |s|^2, |r|^2);
// w = D_c^dag u with the updates in its epilogue.  |r|^2 is that of the
// current r, so convergence is seen one stencil later than in the textbook
// form, with the same iteration count.
// No barrier other than the exchange:
// s and u, the two vectors other CTAs read, live in epoch-tagged buffers
// (s_i and u_i carry epoch E + i), so a stencil's staging waits for exactly the
// entries it reads and needs no flag or fence; the exchange of the partial
// sums (xch_post_packed / xch_collect_packed: a CTA's three sums in one line)
// publishes and polls with relaxed accesses for the same reason.  A writer can
// never be a whole iteration ahead of a reader of the same entry: it overwrites
// s (u) only after the exchange (the next s staging) that needs the reader's
// partial sums, published after the reader's staging; the partial sums depend
// on the staged values and the overwriting values on the collected sums.
template <bool H16, int TM> __device__ void cgls_body_tag(const CglsArgs& a, CglsCta<H16, TM>& c) {
    unsigned int ex = a.epoch0;           // exchange epochs
    const unsigned int E = a.epoch0;      // tag epoch of s_0 and u_0
    float* shr = reinterpret_cast<float*>(c.xs + (size_t)a.sh.nx_max * c.K);
    unsigned long long* ts = a.tag;                                  // s: [Vc * nc][2]
    unsigned long long* tu = a.tag + 2 * (size_t)a.g.Vc * a.nc;      // u
    // y = 0, r = rc on the own rows; |rc|^2
    float one[1] = {0.f};
    for (int i = threadIdx.x; i < c.nu * c.RU; i += blockDim.x) {
        const int j = i / c.RU, ain = i - j * c.RU, u = c.u0 + j, X = u / c.H;
        const size_t o = (size_t)X * c.nc + (u - X * c.H) * c.RU + ain;
        const float2 v = a.rc[o];
        if (c.ov) {
            c.ov[OV_R * c.ov_n + i] = cx<float>(v.x, v.y);
            c.ov[OV_Y * c.ov_n + i] = cx<float>(0.f, 0.f);
        } else {
            a.r[o] = v;
            a.y[o] = make_float2(0.f, 0.f);
        }
        one[0] += v.x * v.x + v.y * v.y;
    }
    const float rpart0 = one[0];
    xch_post_packed<1>(one, a.xch, ex, shr);
    if (!xch_collect_packed<1>(one, a.xch, ex++, a.err, shr)) return;
    const float rc2 = one[0];
    int it = 0;
    float r2 = rc2;
    if (rc2 > 0.f && a.maxit > 0) {
        CglsPhase ph{};
        float n0 = 0.f, n1 = 0.f;
        // s_0 = D_c^dag rc (rc is the launch's input: no tag needed), own |s_0|^2
        ph.in = a.rc;
        ph.tout = ts;
        ph.etag_out = E;
        ph.own_out = OV_S;
        if (!c.template phase<ST_IN, true, EPI_TAG>(ph, n0, n1)) return;
        float gpart = n0, rpart = rpart0;
        float gamma_old = 0.f, alpha_old = 0.f;
        for (int i = 0;; ++i) {
            ph = CglsPhase{};
            ph.tin = ts;
            ph.etag = E + (unsigned int)i;
            ph.tout = tu;
            ph.etag_out = E + (unsigned int)i;
            ph.own_out = OV_U;
            n0 = 0.f; n1 = 0.f;
            if (!c.template phase<ST_TAG, false, EPI_TAG>(ph, n0, n1)) return;   // u = D_c s
            // publish (|u|^2, |s|^2, |r|^2) now and collect the sums only after the
            // products of the second stencil, which do not depend on them: the
            // exchange's latency hides behind w = D_c^dag u
            float three[3] = {n0, gpart, rpart};
            const unsigned int ex_i = ex++;
            xch_post_packed<3>(three, a.xch, ex_i, shr);
            float gamma = 0.f, alpha = 0.f;
            ph = CglsPhase{};
            ph.tin = tu;
            ph.etag = E + (unsigned int)i;
            ph.ts = ts; ph.tu = tu;
            ph.cp = a.p; ph.cz = a.p1; ph.cq = a.q; ph.cy = a.y; ph.cr = a.r;
            ph.etag_out = E + (unsigned int)i + 1u;
            ph.first = (i == 0);
            auto pre = [&]() -> int {
                if (!xch_collect_packed<3>(three, a.xch, ex_i, a.err, shr)) return -1;
                const float delta = three[0];
                gamma = three[1];
                r2 = three[2];
                it = i;
                if ((i > 0 && r2 <= a.tol2 * rc2) || i >= a.maxit) return 0;
                const float beta = i > 0 ? gamma / gamma_old : 0.f;
                const float den = i > 0 ? delta - beta * gamma / alpha_old : delta;
                if (!(gamma > 0.f) || !(den > 0.f)) return 0;
                alpha = gamma / den;
                ph.alpha = alpha;
                ph.beta = beta;
                return 1;
            };
            n0 = 0.f; n1 = 0.f;
            if (!c.template phase<ST_TAG, true, EPI_CG_TAG>(ph, n0, n1, pre)) return;   // w = D_c^dag u, updates
            if (ph.stop) break;
            gpart = n0;
            rpart = n1;
            gamma_old = gamma;
            alpha_old = alpha;
        }
    }
    if (c.ov) {   // the solution (and residual) of the own rows back to global memory
        __syncthreads();
        for (int i = threadIdx.x; i < c.nu * c.RU; i += blockDim.x) {
            const int j = i / c.RU, ain = i - j * c.RU, u = c.u0 + j, X = u / c.H;
            const size_t o = (size_t)X * c.nc + (u - X * c.H) * c.RU + ain;
            const cx<float> y = c.ov[OV_Y * c.ov_n + i], r = c.ov[OV_R * c.ov_n + i];
            a.y[o] = make_float2(y.r, y.i);
            a.r[o] = make_float2(r.r, r.i);
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

// Latency probes (see CGLS_PROBE_*): maxit rounds of the tagged form's two
// stencils (u = D_c s, s' = D_c^dag u, tagged staging and emission, values
// unnormalised and unused) or of its three-value exchange.  Same epochs and
// reader/writer ordering as the solver: a CTA rewrites s (u) only after staging
// the neighbour entries of u (s) that the neighbour writes after reading it.
template <bool H16, int TM> __device__ void cgls_probe(const CglsArgs& a, CglsCta<H16, TM>& c) {
    float* shr = reinterpret_cast<float*>(c.xs + (size_t)a.sh.nx_max * c.K);
    const unsigned int E = a.epoch0;
    if (a.form == CGLS_PROBE_EXCHANGE) {
        for (int i = 0; i < a.maxit; ++i) {
            float three[3] = {1.f, 1.f, 1.f};
            xch_post_packed<3>(three, a.xch, E + (unsigned int)i, shr);
            if (!xch_collect_packed<3>(three, a.xch, E + (unsigned int)i, a.err, shr)) return;
        }
        return;
    }
    unsigned long long* ts = a.tag;
    unsigned long long* tu = a.tag + 2 * (size_t)a.g.Vc * a.nc;
    CglsPhase ph{};
    float n0 = 0.f, n1 = 0.f;
    ph.in = a.rc;
    ph.tout = ts;
    ph.etag_out = E;
    ph.own_out = OV_S;
    if (!c.template phase<ST_IN, true, EPI_TAG>(ph, n0, n1)) return;
    for (int i = 0; i < a.maxit; ++i) {
        ph = CglsPhase{};
        ph.tin = ts; ph.etag = E + (unsigned int)i;
        ph.tout = tu; ph.etag_out = E + (unsigned int)i; ph.own_out = OV_U;
        if (!c.template phase<ST_TAG, false, EPI_TAG>(ph, n0, n1)) return;
        ph = CglsPhase{};
        ph.tin = tu; ph.etag = E + (unsigned int)i;
        ph.tout = ts; ph.etag_out = E + (unsigned int)i + 1u; ph.own_out = OV_S;
        if (!c.template phase<ST_TAG, true, EPI_TAG>(ph, n0, n1)) return;
    }
}

template <bool H16, int TM> __global__ void __launch_bounds__(kCglsThreads, 1) k_cgls_onchip(CglsArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    CglsCta<H16, TM> c(a, smem_raw);
    c.start();
    if (a.form == CGLS_CG_TAGGED)
        cgls_body_tag<H16, TM>(a, c);
    else if (a.form == CGLS_PROBE_STENCILS || a.form == CGLS_PROBE_EXCHANGE)
        cgls_probe<H16, TM>(a, c);
    else
        cgls_body<H16, TM>(a, c);
    c.drain();   // no copy may still be writing shared memory, and no TMEM stays allocated, when the CTA exits
}

// ---------------------------------------------------------------- operator packing
// Au[u = X*H + h][d][b][a - h*RU] from the FP64 operator A[X][d][b][a]; for
// FP16 one scale per (X, d) block, su = max |Re|, |Im| over the block.
template <bool H16> __global__ void k_pack_units(void* Au, float* su, const double2* __restrict__ A, int nc, int RU) {
    __shared__ double sh[33];
    const size_t blk = blockIdx.x, nn = (size_t)nc * nc;
    const int X = (int)(blk / 9), d = (int)(blk % 9), H = nc / RU;
    const double2* Ab = A + blk * nn;
    double inv = 1.0;
    if (H16) {
        double mx = 0;
        for (size_t i = threadIdx.x; i < nn; i += blockDim.x) mx = fmax(mx, fmax(fabs(Ab[i].x), fabs(Ab[i].y)));
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
            sh[32] = m > 0 ? m : 1.0;
            su[blk] = (float)sh[32];
        }
        __syncthreads();
        inv = 1.0 / (double)(float)sh[32];
    }
    for (size_t i = threadIdx.x; i < nn; i += blockDim.x) {
        const int b = (int)(i / nc), arow = (int)(i % nc), h = arow / RU, ain = arow - h * RU;
        const size_t dst = ((((size_t)X * H + h) * 9 + d) * nc + b) * RU + ain;
        if (H16)
            reinterpret_cast<__half2*>(Au)[dst] = __floats2half2_rn((float)(Ab[i].x * inv), (float)(Ab[i].y * inv));
        else
            reinterpret_cast<float2*>(Au)[dst] = make_float2((float)Ab[i].x, (float)Ab[i].y);
    }
}
void coarse_pack_units(void* Au, float* su, const double2* A, int nc, int ru, int Vc, bool h16, cudaStream_t st) {
    note_launch();
    if (h16)
        k_pack_units<true><<<Vc * 9, 256, 0, st>>>(Au, su, A, nc, ru);
    else
        k_pack_units<false><<<Vc * 9, 256, 0, st>>>(Au, su, A, nc, ru);
}

// ---------------------------------------------------------------- shape and launch
namespace {
struct DevLimits {
    int sms = 0, smem = 0, dev = -1;
};
constexpr int kCglsDevs = 16;
// SM count and opt-in shared memory of the current device, looked up once per
// device (atomic slots: host threads calling at once see 0 or the final value)
DevLimits dev_limits() {
    static std::atomic<int> c_sms[kCglsDevs], c_smem[kCglsDevs];
    DevLimits l;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kCglsDevs) return l;
    l.dev = dev;
    l.sms = c_sms[dev].load(std::memory_order_acquire);
    l.smem = c_smem[dev].load(std::memory_order_acquire);
    if (l.sms == 0 || l.smem == 0) {
        cudaDeviceGetAttribute(&l.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&l.smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        c_smem[dev].store(l.smem, std::memory_order_release);
        c_sms[dev].store(l.sms, std::memory_order_release);
    }
    return l;
}
size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }
// tensor-core shape (tm 2): sets own_off, bt_off, mma_lbo, rop_off, rem_max
// from the end `off` of the common regions and returns the padded total
size_t mma_smem(size_t off, CglsShape& s, int K, int smem_optin) {
    const int rows = s.nu_max * s.ru;
    s.own_off = (int)off;
    off = round_up(off + (size_t)OV_COUNT * rows * 8, 128);
    s.bt_off = (int)off;
    s.mma_lbo = kMmaLbo;
    off += (size_t)(K / 4) * kMmaLbo;
    off = round_up(off, 16);
    s.rop_off = (int)off;
    s.rem_max = std::max(0, rows - kMmaRows);
    s.mma_acc = std::min(kMmaMaxAcc, (512 - 32 * ((K + 31) / 32)) / kMmaN);
    off += (size_t)s.rem_max * K * 4;
    return std::max(off, (size_t)smem_optin / 2 + 4096);
}
}  // namespace

// Pick the rows per unit RU (a divisor of nc, a multiple of 4, with RU * element
// bytes a multiple of 16, RU >= 8 when nc allows) that minimises the rows of
// the busiest CTA.  mode CGLS_AUTO: the operator in tensor memory when every
// thread's share fits its 128 columns, else in shared memory when a CTA's units
// fit there (none: false, the caller uses the register-streaming kernel);
// CGLS_SMEM: shared memory only; CGLS_STREAM: streamed through two one-unit
// slot groups by about a third as many CTAs as units (several waves per phase,
// so the ring wraps within every phase), whatever the size.
bool cgls_shape(int nc, int Vc, bool h16, int mode, CglsShape* out) {
    const DevLimits lim = dev_limits();
    if (lim.sms <= 0 || lim.smem <= 2048 || nc < 4 || (nc & 1)) return false;
    const size_t budget = (size_t)lim.smem - 1024;   // leave room for the kernel's static shared memory
    const int esz = h16 ? 4 : 8, T = kCglsThreads;
    const int qpc = h16 ? 8 : 4;                     // row quads per 32-column TMEM chunk
    bool found = false;
    long long best = 0;
    for (int ru = nc; ru >= 4; --ru) {
        if (nc % ru || ru % 4 || (ru * esz) % 16 || (ru < 8 && ru != nc && nc >= 8)) continue;
        CglsShape s{};
        const int H = nc / ru, K = 9 * nc;
        const long long NU = (long long)Vc * H;
        const int G = (int)std::min<long long>(lim.sms, NU);
        s.ru = ru;
        s.grid = G;
        s.nu_max = (int)((NU + G - 1) / G);
        s.nx_max = std::min(Vc, (s.nu_max - 1 + H - 1) / H + 1);
        const size_t ub = (size_t)9 * nc * ru * esz;
        s.stride = (int)(round_up(ub, 128) + (ru * esz) % 128);
        // one reduction buffer of (rows x row splits) <= 4T entries
        s.red_n = std::max(4 * T, s.nu_max * ru);
        size_t off = round_up(256 + (size_t)s.red_n * 8 + (size_t)s.nx_max * 9 * nc * 8 + kXchScratch * 4, 128);
        long long score;
        const int quads = s.nu_max * ru / 4;
        const int ks_min = quads <= T ? T / quads : 0;
        const int chunks = ks_min ? (((K + ks_min - 1) / ks_min) + qpc - 1) / qpc : 1 << 20;
        if (mode == CGLS_STREAM) {
            s.grid = (int)std::min<long long>(lim.sms, (NU + 2) / 3);
            s.nu_max = (int)((NU + s.grid - 1) / s.grid);
            s.nx_max = std::min(Vc, (s.nu_max - 1 + H - 1) / H + 1);
            s.resident = 0;
            s.red_n = std::max(4 * T, ru);   // two reduction buffers (consecutive waves)
            off = round_up(256 + 2 * (size_t)s.red_n * 8 + (size_t)s.nx_max * 9 * nc * 8 + kXchScratch * 4, 128);
            if (off + 2 * (size_t)s.stride > budget) continue;
            s.groups = 2;
            s.wave = 1;
            s.slots = 2;
            score = (long long)s.nu_max * ru;
        } else if (mode == CGLS_AUTO && h16 && K % 8 == 0 && K <= 480 && s.nx_max <= kMmaAgg &&
                   s.nx_max * K <= kStageRegs * T && s.nu_max * ru - kMmaRows <= kMmaRemWarps &&
                   mma_smem(off, s, K, lim.smem) <= budget) {
            // the operator in tensor memory, products on the tensor cores (same
            // padding past half an SM as below)
            s.tm = 2;
            s.resident = 1;
            s.slots = 0;
            s.wave = s.nu_max;
            s.groups = 1;
            off = mma_smem(off, s, K, lim.smem);
            score = (long long)s.nu_max * ru;
        } else if ((mode == CGLS_AUTO || mode == CGLS_TMEM_CORES) && chunks <= 4 && off <= budget) {
            // the operator in tensor memory; shared memory padded past half an SM
            // so that no second CTA of this kernel (and no second all-column TMEM
            // allocation) shares the SM.  Padding to the whole SM would also keep
            // out CTAs of other kernels, but the L1 it leaves is then too small:
            // measured 10.47 against 10.20 us per CG iteration at 16^3x32.  TMEM
            // kernels of this library on different streams are instead ordered on
            // the host (TmemOrder).
            s.tm = 1;
            s.tm_chunks = chunks;
            s.resident = 1;
            s.slots = 0;
            s.wave = s.nu_max;
            s.groups = 1;
            // the own-row vectors of the tagged form after the exchange scratch
            s.own_off = (int)off;
            off = std::max(off + (size_t)OV_COUNT * s.nu_max * ru * 8, (size_t)lim.smem / 2 + 4096);
            if (off > budget) continue;
            score = (long long)s.nu_max * ru + (mode == CGLS_AUTO ? (1LL << 38) : 0);   // tensor-core shapes first
        } else if (mode != CGLS_TMEM_CORES && off + (size_t)s.nu_max * s.stride <= budget) {
            s.resident = 1;
            s.slots = s.nu_max;
            s.wave = s.nu_max;
            s.groups = 1;
            score = (long long)s.nu_max * ru + (mode == CGLS_AUTO ? (1LL << 40) : 0);   // TMEM shapes first
        } else {
            // the operator would have to stream by waves of a few units, each with a
            // CTA barrier and reduction: measured slower than the register-streaming
            // kernel, so that kernel is used instead
            continue;
        }
        s.slot_off = (int)off;
        s.smem = off + (size_t)s.slots * s.stride;
        if (!found || score < best) {
            *out = s;
            best = score;
            found = true;
        }
    }
    return found;
}

cudaError_t cgls_onchip(const CglsArgs& args, cudaStream_t st) {
    const bool h16 = args.su != nullptr, tm = args.sh.tm != 0;
    const int tmk = args.sh.tm;
    if (tmk < 0 || tmk > 2 || (tmk == 2 && !h16)) return cudaErrorInvalidValue;
    const void* fns[2][3] = {{(const void*)k_cgls_onchip<false, 0>, (const void*)k_cgls_onchip<false, 1>, nullptr},
                             {(const void*)k_cgls_onchip<true, 0>, (const void*)k_cgls_onchip<true, 1>,
                              (const void*)k_cgls_onchip<true, 2>}};
    const void* fn = fns[h16][tmk];
    static std::atomic<bool> attr[kCglsDevs][2][3];   // per device: the attribute is set on the current one
    const DevLimits lim = dev_limits();
    if (lim.dev < 0) return cudaErrorInvalidDevice;
    if (!attr[lim.dev][h16][tmk].load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim.smem - 1024);
        if (e != cudaSuccess) return e;
        attr[lim.dev][h16][tmk].store(true, std::memory_order_release);
    }
    if (((args.form == CGLS_CG_TAGGED || args.form == CGLS_PROBE_STENCILS) && !args.tag) || args.sh.smem > (size_t)lim.smem - 1024 || args.sh.grid <= 0 ||
        args.sh.grid > lim.sms ||
        args.sh.grid > kXchMaxGrid || 2 * args.sh.grid > kCglsThreads)
        return cudaErrorInvalidValue;
    int per = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kCglsThreads, args.sh.smem);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
    if (tm && per > 1) return cudaErrorInvalidValue;   // two CTAs on an SM would both ask for all of its TMEM
    CglsArgs a = args;
    void* params[] = {&a};
    if (!tm) {
        note_launch();
        return cudaLaunchCooperativeKernel(fn, dim3(a.sh.grid), dim3(kCglsThreads), params, a.sh.smem, st);
    }
    TmemOrder order(st);
    if (order.error() != cudaSuccess) return order.error();
    note_launch();
    e = cudaLaunchCooperativeKernel(fn, dim3(a.sh.grid), dim3(kCglsThreads), params, a.sh.smem, st);
    if (e != cudaSuccess) return e;
    return order.launched();
}

}  // namespace wmg

// ---------------------------------------------------------------- ordering of TMEM kernels
// A CTA's tcgen05.alloc waits, without a time limit, until the SM has the
// columns it asks for.  The on-chip CG takes all 512 columns of each SM, the
// tensor-core stencil up to 256 per CTA: if one of them ran on an SM while the
// other held columns there, the allocation would wait for the holder to end.
// Both kernels always end on their own (every other wait in them is bounded),
// but so that they never even share an SM, this process's launches of them
// are ordered: an event is recorded on the stream right after each launch,
// and a launch on another stream than the previous one first makes its stream
// wait for that event.  Launches on one stream are ordered anyway; a stream
// being captured into a graph is left alone (the graph is replayed on the
// stream that issues the other TMEM launches).
namespace wmg {
namespace {
std::mutex g_tmem_mutex;
cudaStream_t g_tmem_last = nullptr;
bool g_tmem_any = false;
int g_tmem_dev = -1;
cudaEvent_t g_tmem_event[16] = {};
}  // namespace

TmemOrder::TmemOrder(cudaStream_t st) : st_(st), lock_(g_tmem_mutex) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    err_ = cudaStreamIsCapturing(st, &cs);
    if (err_ != cudaSuccess) return;
    skip_ = cs != cudaStreamCaptureStatusNone;
    if (skip_) return;
    err_ = cudaGetDevice(&dev_);
    if (err_ != cudaSuccess) return;
    if (dev_ < 0 || dev_ >= 16) { err_ = cudaErrorInvalidDevice; return; }
    if (!g_tmem_event[dev_]) {
        err_ = cudaEventCreateWithFlags(&g_tmem_event[dev_], cudaEventDisableTiming);
        if (err_ != cudaSuccess) return;
    }
    if (g_tmem_any && g_tmem_dev == dev_ && g_tmem_last != st) err_ = cudaStreamWaitEvent(st, g_tmem_event[dev_], 0);
}
cudaError_t TmemOrder::launched() {
    if (err_ != cudaSuccess || skip_) return err_;
    cudaError_t e = cudaEventRecord(g_tmem_event[dev_], st_);
    if (e == cudaSuccess) {
        g_tmem_any = true;
        g_tmem_dev = dev_;
        g_tmem_last = st_;
    }
    return e;
}
}  // namespace wmg

// ---------------------------------------------------------------- bounded-wait check
namespace wmg {
// Drives one of the library's device-side waits into a configuration that
// cannot complete, with a short poll limit, so that a test can check that the
// wait gives up, raises the error flag and returns (the kernel then exits
// normally and the context stays usable).  Buffers (all zeroed by the caller):
// words >= 2 * kXchMaxNV * (G + 1) * kXchPad 64-bit words; ctr >= 3 uints;
// err 1 int.  kind 0: epoch exchange expecting G + 1 publishing CTAs (slot G is
// never written); 1: counter barrier expecting G + 1 arrivals; 2: mbarrier
// transaction of 16 bytes that no copy completes; 3: epoch-tagged entry never
// stored with the awaited epoch.
__global__ void k_wait_probe(int kind, unsigned long long* words, unsigned int* ctr, int* err, long long limit) {
    __shared__ float sc[kXchMaxNV * (32 + 64 + 2)];
    __shared__ __align__(8) uint64_t bar;
    const int G = gridDim.x;
    if (kind == 0) {
        float v[1] = {1.f};
        xch_allreduce<1>(v, words, 1u, err, sc, G + 1, limit);
    } else if (kind == 1) {
        grid_sync(ctr, ctr + 1, (unsigned int)G + 1u, err, limit);
    } else if (kind == 2) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
            mbar_expect_tx(&bar, 16);
            if (!mbar_wait(&bar, 0, limit)) atomicExch(err, 1);
        }
    } else if (kind == 3) {
        if (threadIdx.x == 0) {
            float2 v;
            tag_wait(words, 5u, err, v, limit);
        }
    }
}

cudaError_t wait_probe(int kind, int G, unsigned long long* words, unsigned int* ctr, int* err, long long limit,
                       cudaStream_t st) {
    if (kind < 0 || kind > 3 || G < 1 || G > 64 || limit < 1) return cudaErrorInvalidValue;
    note_launch();
    k_wait_probe<<<G, 128, 0, st>>>(kind, words, ctr, err, limit);
    return cudaGetLastError();
}
}  // namespace wmg

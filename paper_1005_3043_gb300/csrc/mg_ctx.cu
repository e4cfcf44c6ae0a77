// Context, solver drivers and the C-ABI of include/wilson_mg.h.
//
// The solve path (flexible GCR, Sec. III) runs its inner work in precision T
// (double or float): the V(0,n) cycle (restriction, coarse CGNR, prolongation,
// MR smoothing) and the Krylov basis.  The solution x and the true residual
// b - D x are kept in FP64.  Host code only sequences kernels; scalars stay on
// the device and are read back at convergence checks.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wilson_mg.h"
#include "mg_launch.h"

using namespace wmg;

std::atomic<long long>& wmg::launch_counter() {
    static std::atomic<long long> c{0};
    return c;
}

namespace {

struct CoarseLevel {
    int nv = 0, nc = 0, cap = 0;
    double2* P64 = nullptr;   // [X][2][nv][6][Vb]
    float2* P32 = nullptr;
    double2* A64 = nullptr;   // [X][9][nc][nc] column-major blocks
    float2* A32 = nullptr;
    __half* Aemb = nullptr;   // FP16 tensor-core embedding of A64 (batched path), built on demand
    bool emb_valid = false;
    __half2* A16 = nullptr;   // FP16 copy with per-block scales s16 (FP16-storage mode), built on demand
    float* s16 = nullptr;
    bool a16_valid = false;
    void* Au = nullptr;       // operator in CGLS units (FP32 or FP16), built on demand
    float* su = nullptr;      // FP16 unit scales [X][d]
    size_t au_bytes = 0;
    bool au_valid = false, au_h16 = false;
    int au_mode = 0;
    CglsShape au_shape{};
    double mass = 0.0;
    bool valid = false;
};

// Workspace of the batched (multi-RHS) solve, sized for npad panel columns.
struct BatchWork {
    int npad = 0, nrhs_cap = 0, K = 0, nc = 0;
    float2 *rcB = nullptr, *yB = nullptr, *rB = nullptr, *sB = nullptr, *pB = nullptr, *qB = nullptr;
    double* cgs = nullptr;          // 9 x npad per-RHS CG scalars
    __half* bt = nullptr;           // split operand tiles of the tensor-core stencil
    float* xpart = nullptr;         // Vc x npad
    float* rpart = nullptr;         // kBatchRowChunks x npad
    int* flags = nullptr;           // [0] active columns, [1] error
    int* h_flags = nullptr;         // pinned
    double* h_iters = nullptr;      // pinned, npad
    float2* r32 = nullptr;          // nrhs x n
    float2* Z = nullptr;            // nrhs x K x n
    float2* Pk = nullptr;           // nrhs x K x n
    double2* x64 = nullptr;         // nrhs x n (internal layout)
    double2* b64 = nullptr;         // nrhs x n
    double* scal = nullptr;         // nrhs x S_COUNT
    double* h_scal = nullptr;       // pinned nrhs x S_COUNT
    cudaStream_t cap = nullptr;     // capture stream
    cudaGraphExec_t graph = nullptr;
    long long graph_key[6] = {0, 0, 0, 0, 0, 0};
};

// Workspace of the red-black preconditioned CG (checkerboard layout).
struct EoWork {
    EoGeom e{};
    double2* U64 = nullptr;   // [p][mu][9][Vh]
    float2* U32 = nullptr;    // paired FP32 links
    bool links_valid = false;
    double2 *b = nullptr, *x = nullptr, *res = nullptr, *t = nullptr;   // FP64 full vectors [p][12][Vh]
    void *xe = nullptr, *r = nullptr, *s = nullptr, *p = nullptr, *q = nullptr, *t1 = nullptr;   // inner, [12][Vh]
    int inner_bytes = 0;      // 8: FP32 inner vectors, 16: FP64
};

// The learned setup's network: 4 parallel-transport layers, 1-8-8-8-1 channels.
struct NnState {
    static constexpr int kLayers = 4;
    static constexpr int kCh[kLayers + 1] = {1, 8, 8, 8, 1};
    float2* W[kLayers] = {};    // FP32 weights used by the kernels
    float2* Wt[kLayers] = {};   // their adjoints (input-gradient pass)
    double2* Wm = nullptr;      // FP64 master weights, all layers
    double2 *G = nullptr, *m = nullptr, *v = nullptr;   // gradient and Adam moments
    int off[kLayers + 1] = {};  // complex offsets of the layers in Wm / G
    float2* act = nullptr;      // activations x0..x4: 26 fine vectors
    float2* ga = nullptr;       // gradient of a layer's output (8 fine vectors)
    float2* gb = nullptr;       // gradient of its input
    float2* part = nullptr;     // weight-gradient partial sums
    float2* r = nullptr;        // (1 - P P^dag) v
    float2* cvec = nullptr;     // coarse temporary (cvec_nv prototypes)
    int cvec_nv = 0;
    int step = 0;
    bool ready = false, weights = false;
};
constexpr int NnState::kCh[];

// Work vectors of the three-level method on level 1 (sized for the level-1
// lattice) and of its level-2 coarse solve.
template <typename T> struct L1Work {
    v2<T>*z = nullptr, *res = nullptr, *zero = nullptr, *sv = nullptr, *sz = nullptr;
    v2<T>* gm = nullptr;     // level-1 GMRES basis, gm_k + 1 vectors
    int gm_k = 0;
    v2<T>*crc = nullptr, *cy = nullptr;                      // level-2 right-hand side and solution
    v2<T>*cr = nullptr, *cr1 = nullptr, *cs = nullptr, *cp = nullptr, *cp1 = nullptr, *cq = nullptr;
    unsigned long long* ctag = nullptr;
    bool ready = false;
};

template <typename T> struct Work {
    v2<T>* r = nullptr;    // GCR residual (T == double: aliases the FP64 residual)
    v2<T>* Z = nullptr;    // K_restart preconditioned directions
    v2<T>* Pk = nullptr;   // K_restart orthonormal D z
    v2<T>* vr = nullptr;   // V-cycle residual r - D e
    v2<T>* vq = nullptr;   // MR q = D r
    v2<T>* sv = nullptr;   // setup: prototype being relaxed
    v2<T>* sr = nullptr;   // setup: its residual
    v2<T>* sz = nullptr;   // setup: cycle output
    v2<T>* tin = nullptr;  // operator hooks
    v2<T>* tout = nullptr;
    v2<T>* crc = nullptr;  // coarse vectors
    v2<T>* cy = nullptr;
    v2<T>* cr = nullptr;
    v2<T>* cs = nullptr;
    v2<T>* cp = nullptr;
    v2<T>* cq = nullptr;
    v2<T>* cr1 = nullptr;  // second buffers of the coarse CG
    v2<T>* cp1 = nullptr;
    unsigned long long* ctag = nullptr;   // epoch-tagged s and u of the on-chip coarse CG (T == float)
    v2<T>* gm = nullptr;   // GMRES smoother basis, gm_k + 1 vectors
    int gm_k = 0;
    int cnc = 0;           // coarse dof the coarse vectors are sized for
    bool ready = false;
};

}  // namespace

struct mg_ctx {
    Geom g{};
    mg_params prm{};
    int K = 16;                      // GCR restart capacity
    cudaStream_t st = nullptr;
    std::string err;
    double mass = 0.0;
    bool has_links = false;
    double2* U64 = nullptr;          // links [mu][X][9][Vb]
    float2* U32 = nullptr;
    float2* U32p = nullptr;         // FP32 links in the dslash's paired layout
    double2* b64 = nullptr;          // FP64 fine vectors (internal layout)
    double2* x64 = nullptr;
    double2* r64 = nullptr;
    double2* stage_a = nullptr;      // boundary-layout staging (12 V complex each)
    double2* stage_b = nullptr;
    double2* protos = nullptr;       // prototypes [nv][X][12][Vb] FP64
    double2* protos_t = nullptr;     // truncated set during setup
    double2* protos_stage = nullptr; // boundary layout, nv vectors
    double2* Aself = nullptr;        // coarse-build scratch
    double2* cstage = nullptr;       // coarse staging (FP64)
    int dev = 0;                     // device current at mg_create (owns every buffer and the stream)
    double setup_ms = 0.0;           // device time of the last adaptive setup (CUDA events)
    CoarseLevel full, trunc;
    BatchWork bw;
    EoWork eo;
    // third level (levels == 3)
    Geom g2{};                       // the level-1 lattice cut into level-2 aggregates
    int* cnbr2 = nullptr;            // level-2 neighbour table
    CoarseLevel full2, trunc2;       // P64/P32: level-2 prolongator panels; A64/A32: A2
    double2* protos2 = nullptr;      // level-2 prototypes [nv2][Vc1][2 nv1] FP64
    double2* protos2_t = nullptr;
    L1Work<float> l1f;
    L1Work<double> l1d;
    NnState nn;
    Work<float> wf;
    Work<double> wd;
    Reduce R{};
    double* h_scal = nullptr;        // pinned host copy of the scalars
    int* d_status = nullptr;
    unsigned int* bar = nullptr;     // persistent-kernel barrier: count, generation, error flag
    int* cnbr = nullptr;             // coarse neighbour table [Vc][9]
    unsigned long long* xch = nullptr;   // exchange slots of the on-chip coarse CGLS
    unsigned int xch_epoch = 1;          // next free epoch
    double* scal_s = nullptr;            // scalars of the GMRES smoother (its Hessenberg matrix)
    int coarse_kernel_used = MG_CK_NONE;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void*> allocs;
    // launch timer
    bool prof = false;
    unsigned int prof_mask = 0xFFu;   // classes the launch timer tracks
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> ev_class;      // class of each (start, stop) pair
    double coarse_mark = 0.0;       // S_CG_TOTAL at the last profile read
    bool coarse16 = false;          // MG_FP16 mode: FP16 coarse operator and FP16 fine smoother storage
    uint2* U16 = nullptr;           // FP16 links (built on demand from U32)
    bool u16_valid = false;
    uint2 *h_r = nullptr, *h_q = nullptr;     // FP16 smoother vectors r, q (+ per-site scales)
    uint2* h_basis = nullptr;                 // FP16 GMRES basis, h_bk + 1 vectors (+ site scales)
    float* h_bscale = nullptr;
    int h_bk = 0;
    float *h_sr = nullptr, *h_sq = nullptr;
};

namespace {

const char* kStatusNames[] = {"MG_OK", "MG_ERR_INVALID_ARG", "MG_ERR_NOT_SETUP", "MG_ERR_OOM",
                              "MG_ERR_NOT_CONVERGED", "MG_ERR_NUMERIC", "MG_ERR_TIMEOUT", "MG_ERR_CUDA"};

int fail(mg_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)
#define CKL()                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = cudaGetLastError();                                                      \
        if (e_ != cudaSuccess) return fail(ctx, MG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)
#define TRY(expr)                                                                                 \
    do {                                                                                          \
        int s_ = (expr);                                                                          \
        if (s_ != MG_OK) return s_;                                                               \
    } while (0)

template <typename P> int dalloc(mg_ctx* ctx, P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, MG_ERR_OOM, std::string("cudaMalloc ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    ctx->allocs.push_back(q);
    *p = (P*)q;
    return MG_OK;
}

void dfree(mg_ctx* ctx, void* q) {
    if (!q) return;
    for (size_t i = 0; i < ctx->allocs.size(); ++i)
        if (ctx->allocs[i] == q) { ctx->allocs.erase(ctx->allocs.begin() + i); break; }
    cudaFree(q);
}

size_t nfine(const mg_ctx* c) { return (size_t)c->g.V * 12; }

int read_scalars(mg_ctx* ctx, int first, int count) {
    CK(cudaMemcpyAsync(ctx->h_scal + first, ctx->R.scal + first, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

// launch timer: a (start, stop) event pair around tracked launches
int prof_mark(mg_ctx* ctx, int cls, bool start) {
    if (!ctx->prof || !((ctx->prof_mask >> cls) & 1u)) return MG_OK;
    if (ctx->ev_used == ctx->ev_pool.size()) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->ev_pool.push_back(e);
    }
    CK(cudaEventRecord(ctx->ev_pool[ctx->ev_used++], ctx->st));
    if (start) ctx->ev_class.push_back(cls);
    return MG_OK;
}
#define PROF_BEGIN(cls) TRY(prof_mark(ctx, cls, true))
#define PROF_END(cls) TRY(prof_mark(ctx, cls, false))

template <typename T> Work<T>& work(mg_ctx* c);
template <> Work<float>& work<float>(mg_ctx* c) { return c->wf; }
template <> Work<double>& work<double>(mg_ctx* c) { return c->wd; }
template <typename T> const v2<T>* links(const mg_ctx* c);
template <> const v2<float>* links<float>(const mg_ctx* c) { return c->U32p; }   // paired layout
template <> const v2<double>* links<double>(const mg_ctx* c) { return c->U64; }
template <typename T> const v2<T>* lvlP(const CoarseLevel& L);
template <> const v2<float>* lvlP<float>(const CoarseLevel& L) { return L.P32; }
template <> const v2<double>* lvlP<double>(const CoarseLevel& L) { return L.P64; }
template <typename T> const v2<T>* lvlA(const CoarseLevel& L);
template <> const v2<float>* lvlA<float>(const CoarseLevel& L) { return L.A32; }
template <> const v2<double>* lvlA<double>(const CoarseLevel& L) { return L.A64; }

template <typename T> int ensure_work(mg_ctx* ctx) {
    Work<T>& w = work<T>(ctx);
    int nc = 2 * ctx->prm.nvec;
    if (w.ready && w.cnc >= nc) return MG_OK;
    size_t n = nfine(ctx), vb = sizeof(v2<T>) * n;
    if (!w.ready) {
        if (std::is_same<T, double>::value) w.r = (v2<T>*)ctx->r64;
        else TRY(dalloc(ctx, &w.r, vb));
        TRY(dalloc(ctx, &w.Z, vb * ctx->K));
        TRY(dalloc(ctx, &w.Pk, vb * ctx->K));
        TRY(dalloc(ctx, &w.vr, vb));
        TRY(dalloc(ctx, &w.vq, vb));
        TRY(dalloc(ctx, &w.sv, vb));
        TRY(dalloc(ctx, &w.sr, vb));
        TRY(dalloc(ctx, &w.sz, vb));
        TRY(dalloc(ctx, &w.tin, vb));
        TRY(dalloc(ctx, &w.tout, vb));
    }
    size_t cb = sizeof(v2<T>) * (size_t)ctx->g.Vc * (nc > 0 ? nc : 2);
    TRY(dalloc(ctx, &w.crc, cb));
    TRY(dalloc(ctx, &w.cy, cb));
    TRY(dalloc(ctx, &w.cr, cb));
    TRY(dalloc(ctx, &w.cs, cb));
    TRY(dalloc(ctx, &w.cp, cb));
    TRY(dalloc(ctx, &w.cq, cb));
    TRY(dalloc(ctx, &w.cr1, cb));
    TRY(dalloc(ctx, &w.cp1, cb));
    if (sizeof(T) == 4) {
        const size_t tb = sizeof(unsigned long long) * 4 * (size_t)ctx->g.Vc * (nc > 0 ? nc : 2);
        TRY(dalloc(ctx, &w.ctag, tb));
        CK(cudaMemsetAsync(w.ctag, 0, tb, ctx->st));   // epoch 0 is never awaited
    }
    w.cnc = nc;
    w.ready = true;
    return MG_OK;
}

int ensure_level(mg_ctx* ctx, CoarseLevel& L, int nv) {
    if (L.cap < nv) {
        // every buffer sized by the capacity goes, the derived ones (FP16 copy,
        // tensor-core embedding) are rebuilt at the new size on demand
        CK(cudaStreamSynchronize(ctx->st));
        for (void* q : {(void*)L.P64, (void*)L.P32, (void*)L.A64, (void*)L.A32, (void*)L.Aemb, (void*)L.A16,
                        (void*)L.s16})
            dfree(ctx, q);
        L.P64 = nullptr; L.P32 = nullptr; L.A64 = nullptr; L.A32 = nullptr;
        L.Aemb = nullptr; L.A16 = nullptr; L.s16 = nullptr;
        L.emb_valid = L.a16_valid = L.au_valid = L.valid = false;
        size_t np = (size_t)nv * nfine(ctx);
        size_t na = (size_t)ctx->g.Vc * 9 * (2 * nv) * (2 * nv);
        TRY(dalloc(ctx, &L.P64, sizeof(double2) * np));
        TRY(dalloc(ctx, &L.P32, sizeof(float2) * np));
        TRY(dalloc(ctx, &L.A64, sizeof(double2) * na));
        TRY(dalloc(ctx, &L.A32, sizeof(float2) * na));
        L.cap = nv;
    }
    L.nv = nv;
    L.nc = 2 * nv;
    return MG_OK;
}

int ensure_protos(mg_ctx* ctx) {
    int nv = ctx->prm.nvec;
    if (ctx->protos) return MG_OK;
    size_t n = nfine(ctx);
    TRY(dalloc(ctx, &ctx->protos, sizeof(double2) * n * nv));
    TRY(dalloc(ctx, &ctx->protos_t, sizeof(double2) * n * nv));
    TRY(dalloc(ctx, &ctx->protos_stage, sizeof(double2) * n * nv));
    TRY(dalloc(ctx, &ctx->Aself, sizeof(double2) * (size_t)ctx->g.Vc * 8 * (2 * nv) * (2 * nv)));
    TRY(dalloc(ctx, &ctx->cstage, sizeof(double2) * (size_t)ctx->g.Vc * 9 * (2 * nv) * (2 * nv)));
    return MG_OK;
}

// P, D_c of a level from nv prototypes (internal FP64 layout)
int build_level(mg_ctx* ctx, CoarseLevel& L, const double2* V, int nv) {
    TRY(ensure_level(ctx, L, nv));
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->st));
    PROF_BEGIN(MG_K_BLOCK_ORTHO);
    block_orthonormalize(L.P64, V, nv, ctx->g, ctx->d_status, ctx->st);
    PROF_END(MG_K_BLOCK_ORTHO);
    CKL();
    int status = 0;
    CK(cudaMemcpyAsync(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (status) {
        L.valid = false;
        return fail(ctx, MG_ERR_NUMERIC, "block orthonormalisation: rank-deficient prototypes in an aggregate");
    }
    size_t np = (size_t)nv * nfine(ctx), na = (size_t)ctx->g.Vc * 9 * L.nc * L.nc;
    convert<double, float>(L.P32, L.P64, np, ctx->st);
    PROF_BEGIN(MG_K_COARSE_BUILD);
    if (ctx->prm.prec_inner != MG_FP64)   // FP32 products, FP64 accumulation
        coarse_build_f32(L.A64, ctx->Aself, L.P32, ctx->U32, nv, ctx->mass, ctx->g, ctx->st);
    else
        coarse_build(L.A64, ctx->Aself, L.P64, ctx->U64, nv, ctx->mass, ctx->g, ctx->st);
    PROF_END(MG_K_COARSE_BUILD);
    CKL();
    convert<double, float>(L.A32, L.A64, na, ctx->st);
    CKL();
    L.mass = ctx->mass;
    L.valid = true;
    L.emb_valid = false;
    L.a16_valid = false;
    L.au_valid = false;
    return MG_OK;
}

// ---------------------------------------------------------------- coarse solve
int ensure_a16(mg_ctx* ctx, CoarseLevel& L, int Vc) {
    if (L.a16_valid) return MG_OK;
    if (L.nc % 4 != 0) return fail(ctx, MG_ERR_INVALID_ARG, "FP16 coarse storage needs an even nvec");
    if (!L.A16) {
        TRY(dalloc(ctx, &L.A16, sizeof(__half2) * (size_t)Vc * 9 * (2 * L.cap) * (2 * L.cap)));
        TRY(dalloc(ctx, &L.s16, sizeof(float) * (size_t)Vc * 9));
    }
    coarse_pack16(L.A16, L.s16, L.A64, L.nc, Vc, ctx->st);
    CKL();
    L.a16_valid = true;
    return MG_OK;
}

// shape mode of the on-chip CGLS for MgParams.coarse_kernel (0, 2, 3, 4)
int cgls_mode(int coarse_kernel) {
    return coarse_kernel == 2 ? CGLS_STREAM : coarse_kernel == 3 ? CGLS_SMEM : coarse_kernel == 4 ? CGLS_TMEM_CORES
                                                                                                    : CGLS_AUTO;
}

// The operator in the unit layout of the on-chip CGLS kernel; false when no
// shape fits this device (the register-streaming kernel is used instead).
int ensure_units(mg_ctx* ctx, CoarseLevel& L, int Vc, bool h16, int mode, bool* ok) {
    *ok = false;
    if (L.au_valid && L.au_h16 == h16 && L.au_mode == mode) {
        *ok = true;
        return MG_OK;
    }
    CglsShape sh{};
    if (!cgls_shape(L.nc, Vc, h16, mode, &sh)) return MG_OK;
    const size_t bytes = (size_t)Vc * 9 * L.nc * L.nc * (h16 ? 4 : 8);
    if (L.au_bytes < bytes) {
        if (L.Au) { dfree(ctx, L.Au); L.Au = nullptr; L.au_bytes = 0; }
        TRY(dalloc(ctx, &L.Au, bytes));
        L.au_bytes = bytes;
    }
    if (h16 && !L.su) TRY(dalloc(ctx, &L.su, sizeof(float) * (size_t)Vc * 9));
    coarse_pack_units(L.Au, h16 ? L.su : nullptr, L.A64, L.nc, sh.ru, Vc, h16, ctx->st);
    CKL();
    L.au_shape = sh;
    L.au_h16 = h16;
    L.au_mode = mode;
    L.au_valid = true;
    *ok = true;
    return MG_OK;
}

template <typename T>
CgnrArgs<T> cgnr_args(const CoarseLevel& L, const Geom& g, const v2<T>* rc, v2<T>* y, v2<T>* r, v2<T>* r1, v2<T>* sv,
                      v2<T>* p, v2<T>* p1, v2<T>* q, double tol, int maxit, double* partials, unsigned int* bar,
                      double* scal) {
    CgnrArgs<T> a;
    a.y = y; a.r = r; a.r1 = r1; a.s = sv; a.p = p; a.p1 = p1; a.q = q;
    a.A = lvlA<T>(L); a.A16 = nullptr; a.s16 = nullptr; a.nbr = nullptr; a.rc = rc; a.nc = L.nc; a.g = g;
    a.tol2 = tol * tol; a.maxit = maxit;
    a.partials = partials; a.bar = bar; a.scal = scal; a.err = (int*)(bar + 2);
    return a;
}

// CGNR on D_c (one persistent cooperative launch).  With iters != nullptr the
// call waits for the result; otherwise the count is only added to
// scal[S_CG_TOTAL] and nothing synchronises.
int clear_epoch_tags(mg_ctx* ctx);

// The coarsest-grid solve of one level: its geometry, neighbour table and CG
// vectors (level 1 -- the two-level method -- or level 2 of the three-level one).
template <typename T> struct CgSys {
    Geom g;            // coarse lattice of the operator (Vc, Lc, xstride)
    const int* nbr;    // its neighbour table [Vc][9]
    v2<T>*cr, *cr1, *cs, *cp, *cp1, *cq;
    unsigned long long* ctag;   // epoch-tagged vectors of the on-chip solver (T == float)
};
template <typename T> CgSys<T> level1_sys(mg_ctx* ctx) {
    Work<T>& w = work<T>(ctx);
    return CgSys<T>{ctx->g, ctx->cnbr, w.cr, w.cr1, w.cs, w.cp, w.cp1, w.cq, w.ctag};
}

template <typename T>
int coarse_solve(mg_ctx* ctx, const CoarseLevel& L, const CgSys<T>& sys, const v2<T>* rc, v2<T>* y, double tol,
                 int maxit, int* iters) {
    CgnrArgs<T> a = cgnr_args<T>(L, sys.g, rc, y, sys.cr, sys.cr1, sys.cs, sys.cp, sys.cp1, sys.cq, tol, maxit,
                                 ctx->R.partials, ctx->bar, ctx->R.scal);
    a.nbr = sys.nbr;
    bool onchip = false;
    if (std::is_same<T, float>::value && ctx->prm.coarse_kernel != 1) {
        CoarseLevel& Lm = const_cast<CoarseLevel&>(L);
        const int mode = cgls_mode(ctx->prm.coarse_kernel);
        TRY(ensure_units(ctx, Lm, sys.g.Vc, ctx->coarse16, mode, &onchip));
    }
    if (onchip) {
        CglsArgs c{};
        c.Au = L.Au; c.su = ctx->coarse16 ? L.su : nullptr; c.nbr = sys.nbr;
        c.rc = (const float2*)a.rc; c.y = (float2*)a.y; c.r = (float2*)a.r; c.r1 = (float2*)a.r1;
        c.s = (float2*)a.s; c.p = (float2*)a.p; c.p1 = (float2*)a.p1; c.q = (float2*)a.q;
        c.nc = L.nc; c.g = sys.g; c.tol2 = (float)(tol * tol); c.maxit = maxit;
        c.scal = ctx->R.scal; c.err = (int*)(ctx->bar + 2);
        c.sh = L.au_shape;
        const unsigned long long reserve = 2ull * (unsigned long long)(maxit > 0 ? maxit : 0) + 4ull;
        if ((unsigned long long)ctx->xch_epoch + reserve >= 0xFFFFFFFFull) {   // 32-bit epochs would wrap
            CK(cudaMemsetAsync(ctx->xch, 0, sizeof(unsigned long long) * kXchWords, ctx->st));
            TRY(clear_epoch_tags(ctx));
            ctx->xch_epoch = 1;
        }
        c.xch = ctx->xch;
        c.epoch0 = ctx->xch_epoch;
        c.form = ctx->prm.coarse_form == 1 ? CGLS_TEXTBOOK : CGLS_CG_TAGGED;
        c.tag = sys.ctag;
        ctx->xch_epoch += (unsigned int)reserve;
        CK(cudaMemsetAsync(ctx->bar, 0, sizeof(unsigned int) * 3, ctx->st));
        PROF_BEGIN(MG_K_COARSE_SOLVE);
        CK(cgls_onchip(c, ctx->st));
        PROF_END(MG_K_COARSE_SOLVE);
        ctx->coarse_kernel_used = c.sh.tm == 2 ? MG_CK_TMEM_MMA : c.sh.tm ? MG_CK_TMEM : c.sh.resident ? MG_CK_SMEM : MG_CK_STREAM;
    } else if (std::is_same<T, float>::value && ctx->coarse16) {
        CoarseLevel& Lm = const_cast<CoarseLevel&>(L);
        TRY(ensure_a16(ctx, Lm, sys.g.Vc));
        a.A16 = Lm.A16;
        a.s16 = Lm.s16;
    }
    if (!onchip) {
        CK(cudaMemsetAsync(ctx->bar, 0, sizeof(unsigned int) * 3, ctx->st));
        PROF_BEGIN(MG_K_COARSE_SOLVE);
        CK(cgnr_persistent<T>(a, ctx->st));
        PROF_END(MG_K_COARSE_SOLVE);
        ctx->coarse_kernel_used = MG_CK_REGISTER;
    }
    if (iters) {
        TRY(read_scalars(ctx, S_CG_RC2, 3));
        unsigned int flags[3];
        CK(cudaMemcpy(flags, ctx->bar, sizeof(flags), cudaMemcpyDeviceToHost));
        if (flags[2]) return fail(ctx, MG_ERR_TIMEOUT, "coarse solve: a grid barrier wait gave up");
        *iters = (int)ctx->h_scal[S_CG_ITERS];
    }
    return MG_OK;
}

// error flag of the persistent kernels (checked once per solve)
int check_timeout(mg_ctx* ctx) {
    unsigned int flags[3];
    CK(cudaMemcpyAsync(flags, ctx->bar, sizeof(flags), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (flags[2]) return fail(ctx, MG_ERR_TIMEOUT, "coarse solve: a grid barrier wait gave up");
    return MG_OK;
}

// ---------------------------------------------------------------- V(0, n) cycle
// Algorithmic bytes per lattice site of one fine operator application: the
// links, one input and one output spinor, each read or written once, in the
// application's storage precision (FP16: 4 x 9 complex link entries in FP16,
// spinors as 12 complex FP16 plus one FP32 site scale).
constexpr double kDslashBytesF64 = 960.0, kDslashBytesF32 = 480.0, kDslashBytesF16 = 144.0 + 2 * 52.0;
template <typename T> constexpr double dslash_site_bytes() {
    return sizeof(T) == 8 ? kDslashBytesF64 : kDslashBytesF32;
}

struct Counters {
    int coarse_iters = 0;
    int matvecs = 0;
    double site_bytes = 0.0;   // sum over applications of the bytes per site
    void fine(int k, double bytes_per_site) {
        matvecs += k;
        site_bytes += k * bytes_per_site;
    }
};

// FP16 links and the FP16 smoother vectors (MG_FP16 mode), built on first use
int ensure_fine16(mg_ctx* ctx) {
    const size_t V = (size_t)ctx->g.V;
    if (!ctx->U16) {
        TRY(dalloc(ctx, &ctx->U16, sizeof(uint2) * 20 * V));
        TRY(dalloc(ctx, &ctx->h_r, sizeof(uint2) * 6 * V));
        TRY(dalloc(ctx, &ctx->h_q, sizeof(uint2) * 6 * V));
        TRY(dalloc(ctx, &ctx->h_sr, sizeof(float) * V));
        TRY(dalloc(ctx, &ctx->h_sq, sizeof(float) * V));
    }
    if (!ctx->u16_valid) {
        links_to_half(ctx->U16, ctx->U32, ctx->g, ctx->st);
        CKL();
        ctx->u16_valid = true;
    }
    return MG_OK;
}

// MG_FP16: whether the smoother stores its spinors and links in FP16.  Its
// dslash is limited by dependent load rounds more than by bytes, so FP16 pays
// only when the FP32 working set would not stay in L2 (measured: 24^3x64
// 103 -> 90 us per dslash with L2 flushed; 16^3x32, L2-resident in a solve,
// 14.7 -> 16.4 us).
bool smoother_fp16(mg_ctx* ctx) {
    if (!ctx->coarse16 || ctx->prm.smoother_fp16 == 2) return false;
    if (ctx->prm.smoother_fp16 == 1) return true;
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    return (double)ctx->g.V * 576.0 > (double)l2;
}

// MG_FP16 with the GMRES smoother: whether its Arnoldi basis is stored in FP16.
// Its Gram-Schmidt passes re-read the whole basis, so FP16 pays when the FP32
// basis ((k + 1) x 96 B per site) would not stay in L2 (smoother_fp16 0), or
// always (1), or never (2).
bool gmres_fp16(mg_ctx* ctx, int k) {
    if (!ctx->coarse16 || ctx->prm.smoother_fp16 == 2) return false;
    if (ctx->prm.smoother_fp16 == 1) return true;
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    return (double)ctx->g.V * 96.0 * (k + 1) > (double)l2;
}

// Post-smoothing of the V(0,n) cycle (Sec. III): r_s = r - D z, then n MR steps
// q = D r_s, alpha = omega <q,r_s>/<q,q>, z += alpha r_s, r_s -= alpha q.  In
// MG_FP16 mode r_s and q are stored in FP16 with a per-site scale and the
// links in FP16 (FP32 arithmetic); z stays in the path's precision.
template <typename T>
int smooth(mg_ctx* ctx, const v2<T>* r, v2<T>* z, const Reduce& R, Counters& cnt) {
    Work<T>& w = work<T>(ctx);
    const size_t n = nfine(ctx);
    const int steps = ctx->prm.smoother_steps;
    if (std::is_same<T, float>::value && ctx->prm.smoother == 1 && steps > 0 && gmres_fp16(ctx, steps)) {
        // GMRES(steps) with the Arnoldi basis in FP16 storage (pairs + site scales): the
        // same algorithm, the basis (steps + 1) x 52 B per site instead of 96 B
        TRY(ensure_fine16(ctx));
        const size_t V = (size_t)ctx->g.V;
        if (ctx->h_bk < steps) {
            if (ctx->h_basis) { dfree(ctx, ctx->h_basis); dfree(ctx, ctx->h_bscale); ctx->h_basis = nullptr; }
            TRY(dalloc(ctx, &ctx->h_basis, sizeof(uint2) * 6 * V * (size_t)(steps + 1)));
            TRY(dalloc(ctx, &ctx->h_bscale, sizeof(float) * V * (size_t)(steps + 1)));
            ctx->h_bk = steps;
        }
        Reduce Rs = R;
        Rs.scal = ctx->scal_s;
        uint2* B = ctx->h_basis;
        float* S = ctx->h_bscale;
        float2* zf = reinterpret_cast<float2*>(z);
        PROF_BEGIN(MG_K_DSLASH);
        dslash_h_xmy(HalfSpinor{B, S}, zf, ctx->U16, reinterpret_cast<const float2*>(r), ctx->g, ctx->mass, ctx->st);
        PROF_END(MG_K_DSLASH);
        PROF_BEGIN(MG_K_KRYLOV);
        h_orth(B, S, ctx->g, 0, Rs, ctx->st);        // no projection for k = 0: |v_0|
        PROF_END(MG_K_KRYLOV);
        for (int j = 0; j < steps; ++j) {
            // v_j is normalised by its norm h_{j,j-1} (|v_0| for j = 0): every reader
            // of the basis scales its site scales by 1 / |v_j| from the scalars
            HalfSpinor out{B + (size_t)(j + 1) * 6 * V, S + (size_t)(j + 1) * V};
            PROF_BEGIN(MG_K_DSLASH);
            dslash_h_plain(out, ConstHalfSpinor(B + (size_t)j * 6 * V, S + (size_t)j * V), ctx->U16, ctx->g, ctx->mass,
                           ctx->st, Rs.scal + S_GMRES_F + j);
            PROF_END(MG_K_DSLASH);
            PROF_BEGIN(MG_K_KRYLOV);
            h_multidot(B, S, ctx->g, j + 1, Rs, ctx->st);
            h_orth(B, S, ctx->g, j + 1, Rs, ctx->st);
            PROF_END(MG_K_KRYLOV);
        }
        PROF_BEGIN(MG_K_KRYLOV);
        gmres_ls(Rs, steps, ctx->prm.omega, ctx->st);
        h_multi_axpy(zf, B, S, ctx->g, steps, Rs, ctx->st);
        PROF_END(MG_K_KRYLOV);
        cnt.fine(steps + 1, kDslashBytesF16);
        return MG_OK;
    }
    if (ctx->prm.smoother == 1 && steps > 0) {
        // one GMRES(steps) application, under-relaxed by omega (Sec. III-IV):
        // Arnoldi with one classical Gram-Schmidt pass per vector, the small
        // least-squares problem on the device, z += omega V y
        if (w.gm_k < steps) {
            if (w.gm) { dfree(ctx, w.gm); w.gm = nullptr; w.gm_k = 0; }
            TRY(dalloc(ctx, &w.gm, sizeof(v2<T>) * n * (size_t)(steps + 1)));
            w.gm_k = steps;
        }
        Reduce Rs = R;
        Rs.scal = ctx->scal_s;
        const v2<T>* U = links<T>(ctx);
        v2<T>* V = w.gm;
        PROF_BEGIN(MG_K_DSLASH);
        dslash<T>(DS_XMY, V, z, U, r, ctx->g, ctx->mass, 0.0, 0, Rs, ctx->st);
        PROF_END(MG_K_DSLASH);
        PROF_BEGIN(MG_K_KRYLOV);
        norm2<T>(V, n, S_GCR_PN2, Rs, ctx->st);
        gmres_normalize<T>(V, n, 0, Rs, ctx->st);
        PROF_END(MG_K_KRYLOV);
        for (int j = 0; j < steps; ++j) {
            PROF_BEGIN(MG_K_DSLASH);
            dslash<T>(DS_PLAIN, V + (size_t)(j + 1) * n, V + (size_t)j * n, U, V, ctx->g, ctx->mass, 0.0, 0, Rs, ctx->st);
            PROF_END(MG_K_DSLASH);
            PROF_BEGIN(MG_K_KRYLOV);
            gcr_multidot<T>(V, n, j + 1, Rs, ctx->st);
            gcr_orth_norm<T>(V, n, j + 1, Rs, ctx->st);
            gmres_normalize<T>(V, n, j + 1, Rs, ctx->st);
            PROF_END(MG_K_KRYLOV);
        }
        PROF_BEGIN(MG_K_KRYLOV);
        gmres_ls(Rs, steps, ctx->prm.omega, ctx->st);
        multi_axpy<T>(z, V, n, steps, Rs, ctx->st);
        PROF_END(MG_K_KRYLOV);
        cnt.fine(steps + 1, dslash_site_bytes<T>());
        return MG_OK;
    }
    if (std::is_same<T, float>::value && smoother_fp16(ctx)) {
        TRY(ensure_fine16(ctx));
        HalfSpinor hr{ctx->h_r, ctx->h_sr}, hq{ctx->h_q, ctx->h_sq};
        float2* zf = reinterpret_cast<float2*>(z);
        PROF_BEGIN(MG_K_DSLASH);
        dslash_h_xmy(hr, zf, ctx->U16, reinterpret_cast<const float2*>(r), ctx->g, ctx->mass, ctx->st);
        PROF_END(MG_K_DSLASH);
        cnt.fine(1, kDslashBytesF16);
        for (int k = 0; k < steps; ++k) {
            PROF_BEGIN(MG_K_DSLASH);
            dslash_h_mrdot(hq, hr, ctx->U16, ctx->g, ctx->mass, ctx->prm.omega, R, ctx->st);
            PROF_END(MG_K_DSLASH);
            PROF_BEGIN(MG_K_KRYLOV);
            mr_update_h(zf, hr, hq, ctx->g, k + 1 < steps, R, ctx->st);
            PROF_END(MG_K_KRYLOV);
            cnt.fine(1, kDslashBytesF16);
        }
        return MG_OK;
    }
    const v2<T>* U = links<T>(ctx);
    PROF_BEGIN(MG_K_DSLASH);
    dslash<T>(DS_XMY, w.vr, z, U, r, ctx->g, ctx->mass, 0.0, 0, R, ctx->st);
    PROF_END(MG_K_DSLASH);
    cnt.fine(1, dslash_site_bytes<T>());
    for (int k = 0; k < steps; ++k) {
        PROF_BEGIN(MG_K_DSLASH);
        dslash<T>(DS_MRDOT, w.vq, w.vr, U, w.vr, ctx->g, ctx->mass, ctx->prm.omega, 0, R, ctx->st);
        PROF_END(MG_K_DSLASH);
        PROF_BEGIN(MG_K_KRYLOV);
        mr_update<T>(z, w.vr, w.vq, n, k + 1 < steps, R, ctx->st);
        PROF_END(MG_K_KRYLOV);
        cnt.fine(1, dslash_site_bytes<T>());
    }
    return MG_OK;
}

// ---------------------------------------------------------------- the third level (Sec. III recursion, Sec. IV W-cycle)
template <typename T> L1Work<T>& l1work(mg_ctx* c);
template <> L1Work<float>& l1work<float>(mg_ctx* c) { return c->l1f; }
template <> L1Work<double>& l1work<double>(mg_ctx* c) { return c->l1d; }

template <typename T> int ensure_l1work(mg_ctx* ctx) {
    L1Work<T>& l = l1work<T>(ctx);
    if (l.ready) return MG_OK;
    const size_t n1 = (size_t)ctx->g.Vc * 2 * ctx->prm.nvec, n2 = (size_t)ctx->g2.Vc * 2 * ctx->prm.nvec2;
    const size_t b1 = sizeof(v2<T>) * n1, b2 = sizeof(v2<T>) * n2;
    TRY(dalloc(ctx, &l.z, b1));
    TRY(dalloc(ctx, &l.res, b1));
    TRY(dalloc(ctx, &l.zero, b1));
    TRY(dalloc(ctx, &l.sv, b1));
    TRY(dalloc(ctx, &l.sz, b1));
    for (v2<T>** q : {&l.crc, &l.cy, &l.cr, &l.cr1, &l.cs, &l.cp, &l.cp1, &l.cq}) TRY(dalloc(ctx, q, b2));
    zero<T>(l.zero, n1, ctx->st);
    if (sizeof(T) == 4) {
        const size_t tb = sizeof(unsigned long long) * 4 * n2;
        TRY(dalloc(ctx, &l.ctag, tb));
        CK(cudaMemsetAsync(l.ctag, 0, tb, ctx->st));   // epoch 0 is never awaited
    }
    l.ready = true;
    return MG_OK;
}
template <typename T> CgSys<T> level2_sys(mg_ctx* ctx) {
    L1Work<T>& l = l1work<T>(ctx);
    return CgSys<T>{ctx->g2, ctx->cnbr2, l.cr, l.cr1, l.cs, l.cp, l.cp1, l.cq, l.ctag};
}

int clear_epoch_tags(mg_ctx* ctx) {
    if (ctx->wf.ctag)
        CK(cudaMemsetAsync(ctx->wf.ctag, 0, sizeof(unsigned long long) * 4 * (size_t)ctx->g.Vc * ctx->wf.cnc, ctx->st));
    if (ctx->l1f.ctag)
        CK(cudaMemsetAsync(ctx->l1f.ctag, 0, sizeof(unsigned long long) * 4 * (size_t)ctx->g2.Vc * 2 * ctx->prm.nvec2,
                           ctx->st));
    return MG_OK;
}

int ensure_level2(mg_ctx* ctx, CoarseLevel& L, int nv2) {
    if (L.cap < nv2) {
        CK(cudaStreamSynchronize(ctx->st));
        for (void* q : {(void*)L.P64, (void*)L.P32, (void*)L.A64, (void*)L.A32, (void*)L.Aemb, (void*)L.A16,
                        (void*)L.s16})
            dfree(ctx, q);
        L.P64 = nullptr; L.P32 = nullptr; L.A64 = nullptr; L.A32 = nullptr;
        L.Aemb = nullptr; L.A16 = nullptr; L.s16 = nullptr;
        L.emb_valid = L.a16_valid = L.au_valid = L.valid = false;
        const size_t np = (size_t)nv2 * ctx->g.Vc * 2 * ctx->prm.nvec;
        const size_t na = (size_t)ctx->g2.Vc * 9 * (2 * nv2) * (2 * nv2);
        TRY(dalloc(ctx, &L.P64, sizeof(double2) * np));
        TRY(dalloc(ctx, &L.P32, sizeof(float2) * np));
        TRY(dalloc(ctx, &L.A64, sizeof(double2) * na));
        TRY(dalloc(ctx, &L.A32, sizeof(float2) * na));
        L.cap = nv2;
    }
    L.nv = nv2;
    L.nc = 2 * nv2;
    return MG_OK;
}

// P2 and A2 = P2^dag D_c P2 of a level-2 set from nv2 level-1 prototypes (FP64)
int build_level2(mg_ctx* ctx, CoarseLevel& L, const double2* V2, int nv2) {
    TRY(ensure_level2(ctx, L, nv2));
    const int nv1 = ctx->prm.nvec;
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->st));
    PROF_BEGIN(MG_K_BLOCK_ORTHO);
    block_orthonormalize_l2(L.P64, V2, nv1, nv2, ctx->g2, ctx->d_status, ctx->st);
    PROF_END(MG_K_BLOCK_ORTHO);
    CKL();
    int status = 0;
    CK(cudaMemcpyAsync(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (status) {
        L.valid = false;
        return fail(ctx, MG_ERR_NUMERIC, "level-2 block orthonormalisation: rank-deficient prototypes in an aggregate");
    }
    const size_t np = (size_t)nv2 * ctx->g.Vc * 2 * nv1, na = (size_t)ctx->g2.Vc * 9 * L.nc * L.nc;
    convert<double, float>(L.P32, L.P64, np, ctx->st);
    PROF_BEGIN(MG_K_COARSE_BUILD);
    CK(coarse_build_l2(L.A64, L.P64, ctx->full.A64, nv1, nv2, ctx->g, ctx->g2, ctx->st));
    PROF_END(MG_K_COARSE_BUILD);
    convert<double, float>(L.A32, L.A64, na, ctx->st);
    CKL();
    L.mass = ctx->mass;
    L.valid = true;
    L.emb_valid = L.a16_valid = L.au_valid = false;
    return MG_OK;
}

// Level-1 post-smoothing: one GMRES(k) application on D_c, scaled by omega
// (Sec. III smoother one level down), on z with the residual r1 - D_c z.
template <typename T> int smooth_l1(mg_ctx* ctx, const v2<T>* r1, v2<T>* z, int k) {
    L1Work<T>& l = l1work<T>(ctx);
    const size_t n1 = (size_t)ctx->g.Vc * ctx->full.nc;
    if (l.gm_k < k) {
        if (l.gm) { dfree(ctx, l.gm); l.gm = nullptr; l.gm_k = 0; }
        TRY(dalloc(ctx, &l.gm, sizeof(v2<T>) * n1 * (size_t)(k + 1)));
        l.gm_k = k;
    }
    Reduce Rs = ctx->R;
    Rs.scal = ctx->scal_s;
    const v2<T>* A1 = lvlA<T>(ctx->full);
    v2<T>* V = l.gm;
    PROF_BEGIN(MG_K_KRYLOV);
    coarse_apply<T>(V, A1, z, ctx->full.nc, false, -1, ctx->g, Rs, ctx->st);   // v_0 = r1 - D_c z
    scale<T>(V, n1, -1.0, ctx->st);
    axpy<T>(V, r1, n1, 1.0, 0.0, ctx->st);
    norm2<T>(V, n1, S_GCR_PN2, Rs, ctx->st);
    gmres_normalize<T>(V, n1, 0, Rs, ctx->st);
    for (int j = 0; j < k; ++j) {
        coarse_apply<T>(V + (size_t)(j + 1) * n1, A1, V + (size_t)j * n1, ctx->full.nc, false, -1, ctx->g, Rs, ctx->st);
        gcr_multidot<T>(V, n1, j + 1, Rs, ctx->st);
        gcr_orth_norm<T>(V, n1, j + 1, Rs, ctx->st);
        gmres_normalize<T>(V, n1, j + 1, Rs, ctx->st);
    }
    gmres_ls(Rs, k, ctx->prm.omega, ctx->st);
    multi_axpy<T>(z, V, n1, k, Rs, ctx->st);
    PROF_END(MG_K_KRYLOV);
    CKL();
    return MG_OK;
}

// M1: one V(0, k1) cycle of levels 1 and 2 on D_c z = r1 (z overwritten):
// r2 = P2^dag r1, CGNR on A2 to coarse_tol, z = P2 y2, level-1 smoothing
template <typename T> int vcycle_l1(mg_ctx* ctx, const CoarseLevel& L2, const v2<T>* r1, v2<T>* z) {
    L1Work<T>& l = l1work<T>(ctx);
    const int nv1 = ctx->prm.nvec;
    PROF_BEGIN(MG_K_RESTRICT);
    restrict_l2<T>(l.crc, lvlP<T>(L2), r1, nv1, L2.nv, ctx->g2, ctx->st);
    PROF_END(MG_K_RESTRICT);
    CKL();
    TRY(coarse_solve<T>(ctx, L2, level2_sys<T>(ctx), l.crc, l.cy, ctx->prm.coarse_tol, ctx->prm.max_coarse, nullptr));
    PROF_BEGIN(MG_K_PROLONG);
    prolong_l2<T>(z, lvlP<T>(L2), l.cy, nv1, L2.nv, ctx->g2, ctx->st);
    PROF_END(MG_K_PROLONG);
    CKL();
    return smooth_l1<T>(ctx, r1, z, ctx->prm.smoother_steps1);
}

// The three-level coarse-grid correction (Sec. IV): cycles1 V-cycles on
// D_c e1 = r1 from e1 = 0, e1 += M1 (r1 - D_c e1)
template <typename T> int kcycle(mg_ctx* ctx, const v2<T>* r1, v2<T>* e1) {
    TRY(ensure_l1work<T>(ctx));
    L1Work<T>& l = l1work<T>(ctx);
    const size_t n1 = (size_t)ctx->g.Vc * ctx->full.nc;
    const v2<T>* A1 = lvlA<T>(ctx->full);
    for (int c = 0; c < ctx->prm.cycles1; ++c) {
        if (c == 0) {
            TRY(vcycle_l1<T>(ctx, ctx->full2, r1, e1));
            continue;
        }
        PROF_BEGIN(MG_K_KRYLOV);
        coarse_apply<T>(l.res, A1, e1, ctx->full.nc, false, -1, ctx->g, ctx->R, ctx->st);   // r1 - D_c e1
        scale<T>(l.res, n1, -1.0, ctx->st);
        axpy<T>(l.res, r1, n1, 1.0, 0.0, ctx->st);
        PROF_END(MG_K_KRYLOV);
        TRY(vcycle_l1<T>(ctx, ctx->full2, l.res, l.z));
        PROF_BEGIN(MG_K_KRYLOV);
        axpy<T>(e1, l.z, n1, 1.0, 0.0, ctx->st);
        PROF_END(MG_K_KRYLOV);
    }
    CKL();
    return MG_OK;
}

// Level-2 adaptive setup (Sec. IV's two-step setup applied to D_c), from the
// random level-1 starts in ctx->protos2
template <typename T> int setup_level2_impl(mg_ctx* ctx) {
    TRY(ensure_l1work<T>(ctx));
    L1Work<T>& l = l1work<T>(ctx);
    const mg_params& p = ctx->prm;
    const int nv2 = p.nvec2, gs = p.setup_group, nt = nv2 - gs;
    const size_t n1 = (size_t)ctx->g.Vc * ctx->full.nc;
    const v2<T>* A1 = lvlA<T>(ctx->full);
    Reduce R = ctx->R;
    // (ii) relaxation on D_c v = 0: setup_init_relax GMRES(1) steps (each one MR step)
    for (int i = 0; i < nv2; ++i) {
        double2* vi = ctx->protos2 + (size_t)i * n1;
        convert<double, T>(l.sv, vi, n1, ctx->st);
        for (int it = 0; it < p.setup_init_relax; ++it) TRY(smooth_l1<T>(ctx, l.zero, l.sv, 1));
        norm2<T>(l.sv, n1, S_NORM_A, R, ctx->st);
        normalize_dev<T>(l.sv, n1, S_NORM_A, R, ctx->st);
        convert<T, double>(vi, l.sv, n1, ctx->st);
    }
    CKL();
    // (iii) groups refined with the truncated two-level method of levels 1 and 2
    if (p.setup_iters > 0 && nt > 0) {
        for (int g0 = 0; g0 < nv2; g0 += gs) {
            int k = 0;
            for (int i = 0; i < nv2; ++i)
                if (i < g0 || i >= g0 + gs)
                    CK(cudaMemcpyAsync(ctx->protos2_t + (size_t)(k++) * n1, ctx->protos2 + (size_t)i * n1,
                                       sizeof(double2) * n1, cudaMemcpyDeviceToDevice, ctx->st));
            TRY(build_level2(ctx, ctx->trunc2, ctx->protos2_t, nt));
            for (int i = g0; i < g0 + gs; ++i) {
                double2* vi = ctx->protos2 + (size_t)i * n1;
                convert<double, T>(l.sv, vi, n1, ctx->st);
                for (int it = 0; it < p.setup_iters; ++it) {
                    coarse_apply<T>(l.res, A1, l.sv, ctx->full.nc, false, -1, ctx->g, R, ctx->st);   // -D_c v
                    scale<T>(l.res, n1, -1.0, ctx->st);
                    TRY(vcycle_l1<T>(ctx, ctx->trunc2, l.res, l.sz));
                    axpy<T>(l.sv, l.sz, n1, 1.0, 0.0, ctx->st);
                    norm2<T>(l.sv, n1, S_NORM_A, R, ctx->st);
                    normalize_dev<T>(l.sv, n1, S_NORM_A, R, ctx->st);
                }
                convert<T, double>(vi, l.sv, n1, ctx->st);
            }
        }
    }
    CKL();
    return build_level2(ctx, ctx->full2, ctx->protos2, nv2);
}

template <typename T>
int vcycle(mg_ctx* ctx, const CoarseLevel& L, const v2<T>* r, v2<T>* z, Counters& cnt) {
    Work<T>& w = work<T>(ctx);
    size_t n = nfine(ctx);
    const v2<T>* U = links<T>(ctx);
    PROF_BEGIN(MG_K_RESTRICT);
    restrict_<T>(w.crc, lvlP<T>(L), r, L.nv, ctx->g, ctx->st);
    PROF_END(MG_K_RESTRICT);
    CKL();
    if (ctx->prm.levels == 3 && &L == &ctx->full)
        TRY(kcycle<T>(ctx, w.crc, w.cy));   // Sec. IV: V-cycles on the intermediate grid
    else
        TRY(coarse_solve<T>(ctx, L, level1_sys<T>(ctx), w.crc, w.cy, ctx->prm.coarse_tol, ctx->prm.max_coarse,
                            nullptr));
    PROF_BEGIN(MG_K_PROLONG);
    prolong<T>(z, lvlP<T>(L), w.cy, L.nv, ctx->g, ctx->st);
    PROF_END(MG_K_PROLONG);
    TRY(smooth<T>(ctx, r, z, ctx->R, cnt));
    CKL();
    return MG_OK;
}

// ---------------------------------------------------------------- flexible GCR
template <typename T> int gcr_solve(mg_ctx* ctx, mg_solve_info* info) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    const mg_params& p = ctx->prm;
    size_t n = nfine(ctx);
    const v2<T>* U = links<T>(ctx);
    Counters cnt;
    int restarts = 0, iters = 0, status = MG_ERR_NOT_CONVERGED;
    CK(cudaEventRecord(ctx->ev0, ctx->st));
    norm2<double>(ctx->b64, n, S_NORM_A, ctx->R, ctx->st);
    zero<double>(ctx->x64, n, ctx->st);
    CK(cudaMemcpyAsync(ctx->r64, ctx->b64, sizeof(double2) * n, cudaMemcpyDeviceToDevice, ctx->st));
    if (!std::is_same<T, double>::value) convert<double, T>(w.r, ctx->r64, n, ctx->st);
    CKL();
    TRY(read_scalars(ctx, S_NORM_A, 1));
    TRY(read_scalars(ctx, S_CG_TOTAL, 1));
    const double coarse_before = ctx->h_scal[S_CG_TOTAL];
    double bnorm = std::sqrt(ctx->h_scal[S_NORM_A]);
    if (!std::isfinite(bnorm)) return fail(ctx, MG_ERR_NUMERIC, "right-hand side is not finite");
    double rel = bnorm > 0 ? 1.0 : 0.0;
    if (bnorm == 0) status = MG_OK;
    double rnorm = bnorm;
    const int K = std::min(p.gcr_restart, ctx->K);
    while (status == MG_ERR_NOT_CONVERGED && iters < p.max_outer) {
        int k = 0;
        double rcycle = rnorm;
        for (; k < K && iters < p.max_outer;) {
            v2<T>* zk = w.Z + (size_t)k * n;
            TRY(vcycle<T>(ctx, ctx->full, w.r, zk, cnt));
            PROF_BEGIN(MG_K_DSLASH);
            dslash<T>(DS_PLAIN, w.Pk + (size_t)k * n, zk, U, zk, ctx->g, ctx->mass, 0.0, 0, ctx->R, ctx->st);
            PROF_END(MG_K_DSLASH);
            cnt.fine(1, dslash_site_bytes<T>());
            PROF_BEGIN(MG_K_KRYLOV);
            if (k > 0) {
                gcr_multidot<T>(w.Pk, n, k, ctx->R, ctx->st);
                gcr_orth_norm<T>(w.Pk, n, k, ctx->R, ctx->st);
            } else {
                norm2<T>(w.Pk, n, S_GCR_PN2, ctx->R, ctx->st);
            }
            gcr_cdot<T>(w.Pk, w.r, n, k, ctx->R, ctx->st);
            gcr_update<T>(w.Pk, w.r, n, k, ctx->R, ctx->st);
            PROF_END(MG_K_KRYLOV);
            CKL();
            TRY(read_scalars(ctx, S_GCR_PN2, 2));
            ++k;
            ++iters;
            double pn = ctx->h_scal[S_GCR_PN2];
            if (!(pn > 0) || !std::isfinite(pn)) {
                status = MG_ERR_NUMERIC;
                break;
            }
            rnorm = std::sqrt(ctx->h_scal[S_GCR_R2]);
            if (rnorm <= p.tol * bnorm) break;
            if (p.delta > 0 && rnorm <= p.delta * rcycle) break;
        }
        if (status == MG_ERR_NUMERIC) break;
        // back substitution R y = c
        TRY(read_scalars(ctx, S_GCR_R, 2 * K_MAX * K_MAX + 2 * K_MAX));
        auto Rr = [&](int j, int kk) { return ctx->h_scal + S_GCR_R + 2 * (kk * K_MAX + j); };
        GcrCoef y{};
        for (int i = k - 1; i >= 0; --i) {
            double sr = ctx->h_scal[S_GCR_C + 2 * i], si = ctx->h_scal[S_GCR_C + 2 * i + 1];
            for (int j = i + 1; j < k; ++j) {
                const double* r = Rr(i, j);
                sr -= r[0] * y.c[2 * j] - r[1] * y.c[2 * j + 1];
                si -= r[0] * y.c[2 * j + 1] + r[1] * y.c[2 * j];
            }
            const double* d = Rr(i, i);
            double den = d[0] * d[0] + d[1] * d[1];
            y.c[2 * i] = (sr * d[0] + si * d[1]) / den;
            y.c[2 * i + 1] = (si * d[0] - sr * d[1]) / den;
        }
        PROF_BEGIN(MG_K_KRYLOV);
        gcr_xupdate<T>(ctx->x64, w.Z, n, k, y, ctx->st);
        PROF_END(MG_K_KRYLOV);
        PROF_BEGIN(MG_K_TRUE_RESIDUAL);
        dslash<double>(DS_XMY_NORM, ctx->r64, ctx->x64, ctx->U64, ctx->b64, ctx->g, ctx->mass, 0.0, S_NORM_B, ctx->R,
                       ctx->st);
        PROF_END(MG_K_TRUE_RESIDUAL);
        cnt.fine(1, kDslashBytesF64);
        CKL();
        TRY(read_scalars(ctx, S_NORM_B, 1));
        ++restarts;
        rnorm = std::sqrt(ctx->h_scal[S_NORM_B]);
        rel = rnorm / bnorm;
        if (!std::isfinite(rel)) { status = MG_ERR_NUMERIC; break; }
        if (rel <= p.tol) status = MG_OK;
        else if (!std::is_same<T, double>::value) convert<double, T>(w.r, ctx->r64, n, ctx->st);
    }
    CK(cudaEventRecord(ctx->ev1, ctx->st));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    TRY(check_timeout(ctx));
    TRY(read_scalars(ctx, S_CG_TOTAL, 1));
    if (info) {
        info->outer_iters = iters;
        info->coarse_iters = (int)(ctx->h_scal[S_CG_TOTAL] - coarse_before);
        info->fine_matvecs = cnt.matvecs;
        info->restarts = restarts;
        info->true_rel_res = rel;
        info->solve_ms = ms;
        info->setup_ms = ctx->setup_ms;
        info->dslash_bytes = cnt.site_bytes * (double)ctx->g.V;
        info->status = status;
    }
    if (status == MG_ERR_NOT_CONVERGED) ctx->err = "max_outer reached";
    if (status == MG_ERR_NUMERIC) ctx->err = "non-finite residual or GCR breakdown";
    return status;
}

// ---------------------------------------------------------------- adaptive setup
// relaxation of prototype v (T) on D v = 0: r = -D v, init_relax MR steps, normalise
template <typename T> int relax_and_normalize(mg_ctx* ctx, v2<T>* v, int steps) {
    Work<T>& w = work<T>(ctx);
    size_t n = nfine(ctx);
    const v2<T>* U = links<T>(ctx);
    dslash<T>(DS_PLAIN, w.sr, v, U, v, ctx->g, ctx->mass, 0.0, 0, ctx->R, ctx->st);
    scale<T>(w.sr, n, -1.0, ctx->st);
    for (int k = 0; k < steps; ++k) {
        dslash<T>(DS_MRDOT, w.vq, w.sr, U, w.sr, ctx->g, ctx->mass, ctx->prm.omega, 0, ctx->R, ctx->st);
        mr_update<T>(v, w.sr, w.vq, n, k + 1 < steps, ctx->R, ctx->st);
    }
    norm2<T>(v, n, S_NORM_A, ctx->R, ctx->st);
    normalize_dev<T>(v, n, S_NORM_A, ctx->R, ctx->st);
    CKL();
    return MG_OK;
}

template <typename T> int setup_impl(mg_ctx* ctx) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    const mg_params& p = ctx->prm;
    size_t n = nfine(ctx);
    int nv = p.nvec;
    const v2<T>* U = links<T>(ctx);
    // (ii) relaxation of every random start
    for (int i = 0; i < nv; ++i) {
        double2* vi = ctx->protos + (size_t)i * n;
        convert<double, T>(w.sv, vi, n, ctx->st);
        TRY(relax_and_normalize<T>(ctx, w.sv, p.setup_init_relax));
        convert<T, double>(vi, w.sv, n, ctx->st);
    }
    CKL();
    // (iii) group refinement with the truncated two-level method
    int gs = p.setup_group, nt = nv - gs;
    if (p.setup_iters > 0 && nt > 0) {
        Counters cnt;
        for (int g0 = 0; g0 < nv; g0 += gs) {
            int k = 0;
            for (int i = 0; i < nv; ++i)
                if (i < g0 || i >= g0 + gs)
                    CK(cudaMemcpyAsync(ctx->protos_t + (size_t)(k++) * n, ctx->protos + (size_t)i * n,
                                       sizeof(double2) * n, cudaMemcpyDeviceToDevice, ctx->st));
            TRY(build_level(ctx, ctx->trunc, ctx->protos_t, nt));
            for (int i = g0; i < g0 + gs; ++i) {
                double2* vi = ctx->protos + (size_t)i * n;
                convert<double, T>(w.sv, vi, n, ctx->st);
                for (int it = 0; it < p.setup_iters; ++it) {
                    dslash<T>(DS_PLAIN, w.sr, w.sv, U, w.sv, ctx->g, ctx->mass, 0.0, 0, ctx->R, ctx->st);
                    scale<T>(w.sr, n, -1.0, ctx->st);
                    TRY(vcycle<T>(ctx, ctx->trunc, w.sr, w.sz, cnt));
                    axpy<T>(w.sv, w.sz, n, 1.0, 0.0, ctx->st);
                    norm2<T>(w.sv, n, S_NORM_A, ctx->R, ctx->st);
                    normalize_dev<T>(w.sv, n, S_NORM_A, ctx->R, ctx->st);
                }
                convert<T, double>(vi, w.sv, n, ctx->st);
                CKL();
            }
        }
    }
    TRY(check_timeout(ctx));
    // (iv) final prolongator and coarse operator
    return build_level(ctx, ctx->full, ctx->protos, nv);
}

int check_params(const int dims[4], const mg_params* p, std::string& why) {
    for (int m = 0; m < 4; ++m) {
        if (dims[m] <= 0 || p->block[m] <= 0 || dims[m] % p->block[m] != 0) {
            why = "lattice extent must be a positive multiple of the block extent";
            return MG_ERR_INVALID_ARG;
        }
    }
    int vb = p->block[0] * p->block[1] * p->block[2] * p->block[3];
    if (6 * vb > 8 * 256) { why = "block volume above 341 sites is not supported"; return MG_ERR_INVALID_ARG; }
    if (p->nvec <= 0 || 2 * p->nvec > 50) { why = "nvec must be in 1..25"; return MG_ERR_INVALID_ARG; }
    if (p->gcr_restart <= 0 || p->gcr_restart > K_MAX) { why = "gcr_restart must be in 1..32"; return MG_ERR_INVALID_ARG; }
    if (p->setup_group <= 0 || p->nvec % p->setup_group != 0) {
        why = "setup_group must divide nvec";
        return MG_ERR_INVALID_ARG;
    }
    if (p->prec_inner != MG_FP64 && p->prec_inner != MG_FP32 && p->prec_inner != MG_FP16) {
        why = "prec_inner must be MG_FP64, MG_FP32 or MG_FP16";
        return MG_ERR_INVALID_ARG;
    }
    if (p->prec_inner == MG_FP16 && p->nvec % 2 != 0) { why = "MG_FP16 needs an even nvec"; return MG_ERR_INVALID_ARG; }
    if (p->coarse_kernel < 0 || p->coarse_kernel > 4) { why = "coarse_kernel must be 0, 1, 2, 3 or 4"; return MG_ERR_INVALID_ARG; }
    if (p->smoother_fp16 < 0 || p->smoother_fp16 > 2) { why = "smoother_fp16 must be 0, 1 or 2"; return MG_ERR_INVALID_ARG; }
    if (p->coarse_form < 0 || p->coarse_form > 1) { why = "coarse_form must be 0 or 1"; return MG_ERR_INVALID_ARG; }
    if (p->smoother < 0 || p->smoother > 1) { why = "smoother must be 0 (MR) or 1 (GMRES)"; return MG_ERR_INVALID_ARG; }
    if (p->smoother == 1 && p->smoother_steps > 16) { why = "GMRES smoother: smoother_steps <= 16"; return MG_ERR_INVALID_ARG; }
    if (p->levels != 2 && p->levels != 3) { why = "levels must be 2 or 3"; return MG_ERR_INVALID_ARG; }
    if (p->levels == 3) {
        int vb2 = 1;
        for (int m = 0; m < 4; ++m) {
            const int lc = dims[m] / p->block[m];
            if (p->block2[m] <= 0 || lc % p->block2[m] != 0) {
                why = "level-1 extent must be a positive multiple of block2";
                return MG_ERR_INVALID_ARG;
            }
            vb2 *= p->block2[m];
        }
        if (p->nvec2 <= 0 || p->nvec2 > 32) { why = "nvec2 must be in 1..32"; return MG_ERR_INVALID_ARG; }
        if (vb2 * p->nvec < p->nvec2) { why = "a level-2 aggregate must hold at least nvec2 dof per chirality"; return MG_ERR_INVALID_ARG; }
        if (p->nvec2 % p->setup_group != 0) { why = "setup_group must divide nvec2"; return MG_ERR_INVALID_ARG; }
        if (p->prec_inner == MG_FP16 && p->nvec2 % 2 != 0) { why = "MG_FP16 needs an even nvec2"; return MG_ERR_INVALID_ARG; }
        if (p->smoother_steps1 < 1 || p->smoother_steps1 > 16) { why = "smoother_steps1 must be in 1..16"; return MG_ERR_INVALID_ARG; }
        if (p->cycles1 < 1 || p->cycles1 > 8) { why = "cycles1 must be in 1..8"; return MG_ERR_INVALID_ARG; }
        if (!build_l2_supported(p->nvec, p->nvec2)) { why = "level-2 build does not support this nvec/nvec2"; return MG_ERR_INVALID_ARG; }
    }
    return MG_OK;
}

// boundary host fine vector -> internal T buffer (through stage_a)
template <typename T> int upload_fine(mg_ctx* ctx, const double* h, v2<T>* d) {
    CK(cudaMemcpyAsync(ctx->stage_a, h, sizeof(double2) * nfine(ctx), cudaMemcpyHostToDevice, ctx->st));
    spinor_to_internal<T>(d, ctx->stage_a, ctx->g, ctx->st);
    CKL();
    return MG_OK;
}
template <typename T> int download_fine(mg_ctx* ctx, const v2<T>* d, double* h) {
    spinor_from_internal<T>(ctx->stage_b, d, ctx->g, ctx->st);
    CKL();
    CK(cudaMemcpyAsync(h, ctx->stage_b, sizeof(double2) * nfine(ctx), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}
template <typename T> int upload_coarse(mg_ctx* ctx, const double* h, v2<T>* d, size_t n) {
    CK(cudaMemcpyAsync(ctx->cstage, h, sizeof(double2) * n, cudaMemcpyHostToDevice, ctx->st));
    convert<double, T>(d, ctx->cstage, n, ctx->st);
    CKL();
    return MG_OK;
}
template <typename T> int download_coarse(mg_ctx* ctx, const v2<T>* d, double* h, size_t n) {
    convert<T, double>(ctx->cstage, d, n, ctx->st);
    CKL();
    CK(cudaMemcpyAsync(h, ctx->cstage, sizeof(double2) * n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

int need_links(mg_ctx* ctx) {
    if (!ctx) return MG_ERR_INVALID_ARG;
    if (!ctx->has_links) return fail(ctx, MG_ERR_NOT_SETUP, "links not set");
    return MG_OK;
}
// level 1 (the coarse operator of the two-level method) is set up
int need_level(mg_ctx* ctx) {
    TRY(need_links(ctx));
    if (!ctx->full.valid) return fail(ctx, MG_ERR_NOT_SETUP, "no coarse operator: call mg_setup or mg_set_null_vectors");
    return MG_OK;
}
// every level of the configured cycle is set up (solves and cycles)
int need_cycle(mg_ctx* ctx) {
    TRY(need_level(ctx));
    if (ctx->prm.levels == 3 && !ctx->full2.valid)
        return fail(ctx, MG_ERR_NOT_SETUP, "levels = 3: call mg_setup_level2 or mg_set_level2_vectors");
    return MG_OK;
}

template <typename T> int hook_dslash(mg_ctx* ctx, const double* in, double* out) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    TRY(upload_fine<T>(ctx, in, w.tin));
    if (std::is_same<T, float>::value && ctx->coarse16) {
        // MG_FP16 (the hook always uses the FP16 storage, whatever smoother_fp16
        // selects for solves): the input rounded to FP16 with its site scale, FP16 links,
        // the output rounded likewise (then widened for the caller)
        TRY(ensure_fine16(ctx));
        HalfSpinor hr{ctx->h_r, ctx->h_sr}, hq{ctx->h_q, ctx->h_sq};
        to_half(hr, reinterpret_cast<const float2*>(w.tin), ctx->g, ctx->st);
        dslash_h_plain(hq, hr, ctx->U16, ctx->g, ctx->mass, ctx->st);
        from_half(reinterpret_cast<float2*>(w.tout), hq, ctx->g, ctx->st);
    } else {
        dslash<T>(DS_PLAIN, w.tout, w.tin, links<T>(ctx), w.tin, ctx->g, ctx->mass, 0.0, 0, ctx->R, ctx->st);
    }
    CKL();
    return download_fine<T>(ctx, w.tout, out);
}
template <typename T> int hook_restrict(mg_ctx* ctx, const double* r, double* rc) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    TRY(upload_fine<T>(ctx, r, w.tin));
    restrict_<T>(w.crc, lvlP<T>(ctx->full), w.tin, ctx->full.nv, ctx->g, ctx->st);
    CKL();
    return download_coarse<T>(ctx, w.crc, rc, (size_t)ctx->g.Vc * ctx->full.nc);
}
template <typename T> int hook_prolong(mg_ctx* ctx, const double* yc, double* e) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    TRY(upload_coarse<T>(ctx, yc, w.cy, (size_t)ctx->g.Vc * ctx->full.nc));
    prolong<T>(w.tout, lvlP<T>(ctx->full), w.cy, ctx->full.nv, ctx->g, ctx->st);
    CKL();
    return download_fine<T>(ctx, w.tout, e);
}
template <typename T> int hook_coarse(mg_ctx* ctx, const double* x, double* y, int dagger) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    size_t n = (size_t)ctx->g.Vc * ctx->full.nc;
    TRY(upload_coarse<T>(ctx, x, w.cp, n));
    coarse_apply<T>(w.cq, lvlA<T>(ctx->full), w.cp, ctx->full.nc, dagger != 0, -1, ctx->g, ctx->R, ctx->st);
    CKL();
    return download_coarse<T>(ctx, w.cq, y, n);
}
template <typename T> int hook_mr(mg_ctx* ctx, double* e, double* r, int nsteps) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    size_t n = nfine(ctx);
    TRY(upload_fine<T>(ctx, e, w.tin));
    TRY(upload_fine<T>(ctx, r, w.tout));
    const v2<T>* U = links<T>(ctx);
    if (std::is_same<T, float>::value && ctx->coarse16) {
        // MG_FP16 (always FP16 storage here): r and q in FP16, e in FP32
        TRY(ensure_fine16(ctx));
        HalfSpinor hr{ctx->h_r, ctx->h_sr}, hq{ctx->h_q, ctx->h_sq};
        to_half(hr, reinterpret_cast<const float2*>(w.tout), ctx->g, ctx->st);
        for (int k = 0; k < nsteps; ++k) {
            dslash_h_mrdot(hq, hr, ctx->U16, ctx->g, ctx->mass, ctx->prm.omega, ctx->R, ctx->st);
            mr_update_h(reinterpret_cast<float2*>(w.tin), hr, hq, ctx->g, true, ctx->R, ctx->st);
        }
        from_half(reinterpret_cast<float2*>(w.tout), hr, ctx->g, ctx->st);
    } else {
        for (int k = 0; k < nsteps; ++k) {
            dslash<T>(DS_MRDOT, w.vq, w.tout, U, w.tout, ctx->g, ctx->mass, ctx->prm.omega, 0, ctx->R, ctx->st);
            mr_update<T>(w.tin, w.tout, w.vq, n, true, ctx->R, ctx->st);
        }
    }
    CKL();
    TRY(download_fine<T>(ctx, w.tin, e));
    return download_fine<T>(ctx, w.tout, r);
}
template <typename T>
int hook_coarse_solve(mg_ctx* ctx, const double* rc, double* y, double tol, int maxit, int* iters, double* rel) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    size_t n = (size_t)ctx->g.Vc * ctx->full.nc;
    TRY(upload_coarse<T>(ctx, rc, w.crc, n));
    int it = 0;
    TRY(coarse_solve<T>(ctx, ctx->full, level1_sys<T>(ctx), w.crc, w.cy, tol, maxit, &it));
    TRY(read_scalars(ctx, S_CG_RC2, 2));
    if (iters) *iters = it;
    if (rel) *rel = ctx->h_scal[S_CG_RC2] > 0 ? std::sqrt(ctx->h_scal[S_CG_R2] / ctx->h_scal[S_CG_RC2]) : 0.0;
    return download_coarse<T>(ctx, w.cy, y, n);
}
template <typename T> int hook_vcycle(mg_ctx* ctx, const double* r, double* z) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    TRY(upload_fine<T>(ctx, r, w.tin));
    Counters cnt;
    TRY(vcycle<T>(ctx, ctx->full, w.tin, w.tout, cnt));
    TRY(check_timeout(ctx));
    return download_fine<T>(ctx, w.tout, z);
}

}  // namespace

// ======================================================================= C-ABI
extern "C" {

int mg_default_params(mg_params* p) {
    if (!p) return MG_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    for (int m = 0; m < 4; ++m) p->block[m] = 4;
    p->nvec = 8;
    p->levels = 2;
    for (int m = 0; m < 4; ++m) p->block2[m] = 2;
    p->nvec2 = 32;
    p->smoother_steps1 = 4;
    p->cycles1 = 2;
    p->setup_init_relax = 10;
    p->setup_iters = 3;
    p->setup_group = 4;
    p->smoother_steps = 4;
    p->omega = 0.9;
    p->gcr_restart = 16;
    p->tol = 1e-10;
    p->coarse_tol = 1e-3;
    p->max_outer = 1000;
    p->max_coarse = 5000;
    p->delta = 0.0;
    p->prec_inner = MG_FP64;
    p->coarse_check = 16;
    return MG_OK;
}

int mg_create(const int dims[4], int t_antiperiodic, const mg_params* p, void* stream, mg_ctx** out) {
    if (!dims || !p || !out) return MG_ERR_INVALID_ARG;
    *out = nullptr;
    std::string why;
    if (check_params(dims, p, why) != MG_OK) return MG_ERR_INVALID_ARG;
    mg_ctx* ctx = new mg_ctx();
    if (cudaGetDevice(&ctx->dev) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return MG_ERR_CUDA;
    }
    ctx->prm = *p;
    ctx->K = p->gcr_restart;
    ctx->st = (cudaStream_t)stream;
    Geom& g = ctx->g;
    for (int m = 0; m < 4; ++m) {
        g.L[m] = dims[m];
        g.B[m] = p->block[m];
        g.Lc[m] = dims[m] / p->block[m];
    }
    g.lstride[0] = 1;
    g.xstride[0] = 1;
    for (int m = 1; m < 4; ++m) {
        g.lstride[m] = g.lstride[m - 1] * g.B[m - 1];
        g.xstride[m] = g.xstride[m - 1] * g.Lc[m - 1];
    }
    g.Vb = g.B[0] * g.B[1] * g.B[2] * g.B[3];
    g.Vc = g.Lc[0] * g.Lc[1] * g.Lc[2] * g.Lc[3];
    g.V = (long long)g.Vb * g.Vc;
    g.tap = t_antiperiodic ? 1 : 0;
    if (p->levels == 3) {   // the level-1 lattice cut into level-2 aggregates
        Geom& h = ctx->g2;
        for (int m = 0; m < 4; ++m) {
            h.L[m] = g.Lc[m];
            h.B[m] = p->block2[m];
            h.Lc[m] = g.Lc[m] / p->block2[m];
        }
        h.lstride[0] = 1;
        h.xstride[0] = 1;
        for (int m = 1; m < 4; ++m) {
            h.lstride[m] = h.lstride[m - 1] * h.B[m - 1];
            h.xstride[m] = h.xstride[m - 1] * h.Lc[m - 1];
        }
        h.Vb = h.B[0] * h.B[1] * h.B[2] * h.B[3];
        h.Vc = h.Lc[0] * h.Lc[1] * h.Lc[2] * h.Lc[3];
        h.V = g.Vc;
        h.tap = 0;   // the t boundary sign lives inside D_c
    }
    size_t n = nfine(ctx);
    int rc = MG_OK;
    if ((rc = dalloc(ctx, &ctx->U64, sizeof(double2) * 36 * (size_t)g.V)) ||
        (rc = dalloc(ctx, &ctx->U32, sizeof(float2) * 36 * (size_t)g.V)) ||
        (rc = dalloc(ctx, &ctx->U32p, sizeof(float2) * 36 * (size_t)g.V)) ||
        (rc = dalloc(ctx, &ctx->b64, sizeof(double2) * n)) || (rc = dalloc(ctx, &ctx->x64, sizeof(double2) * n)) ||
        (rc = dalloc(ctx, &ctx->r64, sizeof(double2) * n)) ||
        (rc = dalloc(ctx, &ctx->stage_a, sizeof(double2) * 36 * (size_t)g.V)) ||
        (rc = dalloc(ctx, &ctx->stage_b, sizeof(double2) * n)) ||
        (rc = dalloc(ctx, &ctx->R.partials, reduce_partial_bytes(g.V))) ||
        (rc = dalloc(ctx, &ctx->R.ticket, sizeof(unsigned int) * 4)) ||
        (rc = dalloc(ctx, &ctx->R.scal, sizeof(double) * S_COUNT)) || (rc = dalloc(ctx, &ctx->d_status, sizeof(int))) ||
        (rc = dalloc(ctx, &ctx->bar, sizeof(unsigned int) * 4)) ||
        (rc = dalloc(ctx, &ctx->cnbr, sizeof(int) * 9 * (size_t)g.Vc)) ||
        (rc = dalloc(ctx, &ctx->xch, sizeof(unsigned long long) * kXchWords)) ||
        (rc = dalloc(ctx, &ctx->scal_s, sizeof(double) * S_COUNT))) {
        mg_destroy(ctx);
        return rc;
    }
    ctx->R.partial_bytes = reduce_partial_bytes(g.V);
    if (cudaMallocHost(&ctx->h_scal, sizeof(double) * S_COUNT) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess ||
        cudaMemsetAsync(ctx->R.ticket, 0, sizeof(unsigned int) * 4, ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->R.scal, 0, sizeof(double) * S_COUNT, ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->bar, 0, sizeof(unsigned int) * 4, ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->xch, 0, sizeof(unsigned long long) * kXchWords, ctx->st) != cudaSuccess ||
        (coarse_neighbour_table(ctx->cnbr, ctx->g, ctx->st), cudaGetLastError()) != cudaSuccess ||
        (p->levels == 3 && (dalloc(ctx, &ctx->cnbr2, sizeof(int) * 9 * (size_t)ctx->g2.Vc) != MG_OK ||
                            (coarse_neighbour_table(ctx->cnbr2, ctx->g2, ctx->st), cudaGetLastError()) != cudaSuccess)) ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess) {
        cudaGetLastError();
        mg_destroy(ctx);
        return MG_ERR_CUDA;
    }
    *out = ctx;
    return MG_OK;
}

void mg_destroy(mg_ctx* ctx) {
    if (!ctx) return;
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    else cudaDeviceSynchronize();
    for (void* q : ctx->allocs) cudaFree(q);
    if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->bw.graph) cudaGraphExecDestroy(ctx->bw.graph);
    if (ctx->bw.cap) cudaStreamDestroy(ctx->bw.cap);
    if (ctx->bw.h_flags) cudaFreeHost(ctx->bw.h_flags);
    if (ctx->bw.h_iters) cudaFreeHost(ctx->bw.h_iters);
    if (ctx->bw.h_scal) cudaFreeHost(ctx->bw.h_scal);
    delete ctx;
}

namespace {
// links (boundary layout, device memory) -> the internal FP64, FP32 and paired
// FP32 copies, on the context stream; every level built on the old links is stale
int load_links(mg_ctx* ctx, const double2* U_dev) {
    links_to_internal<double>(ctx->U64, U_dev, ctx->g, ctx->st);
    convert<double, float>(ctx->U32, ctx->U64, 36 * (size_t)ctx->g.V, ctx->st);
    links_pair(ctx->U32p, ctx->U32, ctx->g, ctx->st);
    CKL();
    ctx->has_links = true;
    ctx->u16_valid = false;
    ctx->eo.links_valid = false;
    ctx->full.valid = false;   // D_c depends on the links
    return MG_OK;
}
}  // namespace

int mg_set_links(mg_ctx* ctx, const double* U) {
    if (!ctx || !U) return MG_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(ctx->stage_a, U, sizeof(double2) * 36 * (size_t)ctx->g.V, cudaMemcpyHostToDevice, ctx->st));
    TRY(load_links(ctx, ctx->stage_a));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

int mg_set_links_device(mg_ctx* ctx, const double* U_dev, void* stream) {
    if (!ctx || !U_dev) return MG_ERR_INVALID_ARG;
    cudaStream_t cs = (cudaStream_t)stream;
    // the context stream waits for the caller's work that produced U_dev ...
    if (cs != ctx->st) {
        CK(cudaEventRecord(ctx->ev1, cs));
        CK(cudaStreamWaitEvent(ctx->st, ctx->ev1, 0));
    }
    TRY(load_links(ctx, (const double2*)U_dev));
    // ... and the caller's stream waits for the conversion, so that work the
    // caller queues after this call may overwrite or free U_dev
    if (cs != ctx->st) {
        CK(cudaEventRecord(ctx->ev1, ctx->st));
        CK(cudaStreamWaitEvent(cs, ctx->ev1, 0));
    }
    return MG_OK;
}

int mg_set_mass(mg_ctx* ctx, double m) {
    if (!ctx) return MG_ERR_INVALID_ARG;
    if (ctx->full.valid) {
        coarse_shift_mass(ctx->full.A64, ctx->full.nc, m - ctx->full.mass, ctx->g, ctx->st);
        convert<double, float>(ctx->full.A32, ctx->full.A64, (size_t)ctx->g.Vc * 9 * ctx->full.nc * ctx->full.nc, ctx->st);
        CKL();
        ctx->full.mass = m;
        ctx->full.emb_valid = false;
        ctx->full.a16_valid = false;
        ctx->full.au_valid = false;
    }
    if (ctx->full2.valid) {   // A2(m) = P2^dag D_c(m) P2 = A2(m0) + (m - m0) I, P2^dag P2 = I
        CoarseLevel& L = ctx->full2;
        coarse_shift_mass(L.A64, L.nc, m - L.mass, ctx->g2, ctx->st);
        convert<double, float>(L.A32, L.A64, (size_t)ctx->g2.Vc * 9 * L.nc * L.nc, ctx->st);
        CKL();
        L.mass = m;
        L.emb_valid = L.a16_valid = L.au_valid = false;
    }
    ctx->mass = m;
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

int mg_set_params(mg_ctx* ctx, const mg_params* p) {
    if (!ctx || !p) return MG_ERR_INVALID_ARG;
    std::string why;
    if (check_params(ctx->g.L, p, why) != MG_OK) return fail(ctx, MG_ERR_INVALID_ARG, why);
    for (int m = 0; m < 4; ++m)
        if (p->block[m] != ctx->prm.block[m]) return fail(ctx, MG_ERR_INVALID_ARG, "block size is fixed at create");
    if (p->nvec != ctx->prm.nvec) return fail(ctx, MG_ERR_INVALID_ARG, "nvec is fixed at create");
    if (p->levels != ctx->prm.levels || p->nvec2 != ctx->prm.nvec2 ||
        (p->levels == 3 && std::memcmp(p->block2, ctx->prm.block2, sizeof(p->block2)) != 0))
        return fail(ctx, MG_ERR_INVALID_ARG, "levels, block2 and nvec2 are fixed at create");
    if (p->gcr_restart > ctx->K) return fail(ctx, MG_ERR_INVALID_ARG, "gcr_restart above the value at create");
    ctx->prm = *p;
    return MG_OK;
}

namespace {
// the adaptive setup from the prototypes' random starts (already in ctx->protos,
// internal layout), timed on the context stream from the event recorded in ev0
int run_setup(mg_ctx* ctx) {
    ctx->coarse16 = ctx->prm.prec_inner == MG_FP16;
    int st = ctx->prm.prec_inner != MG_FP64 ? setup_impl<float>(ctx) : setup_impl<double>(ctx);
    if (st != MG_OK) return st;
    CK(cudaEventRecord(ctx->ev1, ctx->st));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    ctx->setup_ms = ms;
    return MG_OK;
}
}  // namespace

int mg_setup(mg_ctx* ctx, const double* V0) {
    TRY(need_links(ctx));
    if (!V0) return fail(ctx, MG_ERR_INVALID_ARG, "V0 is NULL");
    TRY(ensure_protos(ctx));
    int nv = ctx->prm.nvec;
    size_t n = nfine(ctx);
    CK(cudaEventRecord(ctx->ev0, ctx->st));
    CK(cudaMemcpyAsync(ctx->protos_stage, V0, sizeof(double2) * n * nv, cudaMemcpyHostToDevice, ctx->st));
    for (int i = 0; i < nv; ++i)
        spinor_to_internal<double>(ctx->protos + (size_t)i * n, ctx->protos_stage + (size_t)i * n, ctx->g, ctx->st);
    CKL();
    return run_setup(ctx);
}

int mg_setup_device(mg_ctx* ctx, const double* V0_dev) {
    TRY(need_links(ctx));
    if (!V0_dev) return fail(ctx, MG_ERR_INVALID_ARG, "V0 is NULL");
    TRY(ensure_protos(ctx));
    size_t n = nfine(ctx);
    CK(cudaEventRecord(ctx->ev0, ctx->st));
    for (int i = 0; i < ctx->prm.nvec; ++i)
        spinor_to_internal<double>(ctx->protos + (size_t)i * n, (const double2*)V0_dev + (size_t)i * n, ctx->g, ctx->st);
    CKL();
    return run_setup(ctx);
}

int mg_set_null_vectors(mg_ctx* ctx, const double* V, int nv) {
    TRY(need_links(ctx));
    if (!V || nv != ctx->prm.nvec) return fail(ctx, MG_ERR_INVALID_ARG, "nv must equal params.nvec");
    TRY(ensure_protos(ctx));
    size_t n = nfine(ctx);
    CK(cudaMemcpyAsync(ctx->protos_stage, V, sizeof(double2) * n * nv, cudaMemcpyHostToDevice, ctx->st));
    for (int i = 0; i < nv; ++i)
        spinor_to_internal<double>(ctx->protos + (size_t)i * n, ctx->protos_stage + (size_t)i * n, ctx->g, ctx->st);
    CKL();
    return build_level(ctx, ctx->full, ctx->protos, nv);
}

// ---- the learned setup (gauge-covariant parallel-transport network)
}  // extern "C"
namespace {
constexpr int kNnParams = 20736;   // complex weights: 1152 + 9216 + 9216 + 1152
int ensure_nn(mg_ctx* ctx) {
    NnState& q = ctx->nn;
    if (q.ready) return MG_OK;
    const size_t n = nfine(ctx);
    int o = 0;
    for (int k = 0; k < NnState::kLayers; ++k) {
        q.off[k] = o;
        const int c = NnState::kCh[k] * NnState::kCh[k + 1] * 144;
        TRY(dalloc(ctx, &q.W[k], sizeof(float2) * c));
        TRY(dalloc(ctx, &q.Wt[k], sizeof(float2) * c));
        o += c;
    }
    q.off[NnState::kLayers] = o;
    TRY(dalloc(ctx, &q.Wm, sizeof(double2) * o));
    TRY(dalloc(ctx, &q.G, sizeof(double2) * o));
    TRY(dalloc(ctx, &q.m, sizeof(double2) * o));
    TRY(dalloc(ctx, &q.v, sizeof(double2) * o));
    TRY(dalloc(ctx, &q.act, sizeof(float2) * n * 26));
    TRY(dalloc(ctx, &q.ga, sizeof(float2) * n * 8));
    TRY(dalloc(ctx, &q.gb, sizeof(float2) * n * 8));
    TRY(dalloc(ctx, &q.part, sizeof(float2) * (size_t)nn_wgrad_blocks(ctx->g) * 576 * 16));
    TRY(dalloc(ctx, &q.r, sizeof(float2) * n));
    CK(cudaMemsetAsync(q.m, 0, sizeof(double2) * o, ctx->st));
    CK(cudaMemsetAsync(q.v, 0, sizeof(double2) * o, ctx->st));
    q.ready = true;
    return MG_OK;
}
// FP32 weights and their adjoints from the FP64 master copy
int nn_refresh(mg_ctx* ctx) {
    NnState& q = ctx->nn;
    for (int k = 0; k < NnState::kLayers; ++k) {
        convert<double, float>(q.W[k], q.Wm + q.off[k], (size_t)(q.off[k + 1] - q.off[k]), ctx->st);
        nn_adjoint_weights(q.Wt[k], q.W[k], NnState::kCh[k], NnState::kCh[k + 1], ctx->st);
    }
    CKL();
    return MG_OK;
}
float2* nn_act(mg_ctx* ctx, int k) {   // activation k (channels kCh[k]) inside act
    size_t c = 0;
    for (int j = 0; j < k; ++j) c += NnState::kCh[j];
    return ctx->nn.act + c * nfine(ctx);
}
// x0 = eta (internal FP32, in act), then x1..x4
int nn_forward(mg_ctx* ctx) {
    NnState& q = ctx->nn;
    for (int k = 0; k < NnState::kLayers; ++k)
        CK(nn_layer(nn_act(ctx, k + 1), nn_act(ctx, k), q.W[k], ctx->U32, ctx->g, NnState::kCh[k], NnState::kCh[k + 1],
                    ctx->st));
    return MG_OK;
}
// loss |(1 - P P^dag) v|^2 / |v|^2 of x4 into scal[S_NORM_B] / scal[S_NORM_A] and,
// with grad, the gradient (scaled by gscale) added to G
enum { NN_V2 = S_EO + 10, NN_R2 = S_EO + 11 };
int nn_loss_grad(mg_ctx* ctx, bool grad, double gscale) {
    NnState& q = ctx->nn;
    const size_t n = nfine(ctx);
    const CoarseLevel& L = ctx->full;
    if (q.cvec_nv < L.nv) {   // sized by the current level (nvec may change with mg_set_params)
        if (q.cvec) {
            CK(cudaStreamSynchronize(ctx->st));
            dfree(ctx, q.cvec);
        }
        TRY(dalloc(ctx, &q.cvec, sizeof(float2) * (size_t)ctx->g.Vc * 2 * L.nv));
        q.cvec_nv = L.nv;
    }
    float2* v = reinterpret_cast<float2*>(nn_act(ctx, NnState::kLayers));
    restrict_<float>((v2<float>*)q.cvec, L.P32, (const v2<float>*)v, L.nv, ctx->g, ctx->st);
    prolong<float>((v2<float>*)q.r, L.P32, (const v2<float>*)q.cvec, L.nv, ctx->g, ctx->st);
    scale<float>((v2<float>*)q.r, n, -1.0, ctx->st);
    axpy<float>((v2<float>*)q.r, (const v2<float>*)v, n, 1.0, 0.0, ctx->st);
    norm2<float>((const v2<float>*)v, n, NN_V2, ctx->R, ctx->st);
    norm2<float>((const v2<float>*)q.r, n, NN_R2, ctx->R, ctx->st);
    CKL();
    if (!grad) return MG_OK;
    nn_seed(q.ga, q.r, v, n, ctx->R.scal, NN_V2, NN_R2, ctx->st);
    float2* gout = q.ga;
    float2* gin = q.gb;
    for (int k = NnState::kLayers - 1; k >= 0; --k) {
        const int ci = NnState::kCh[k], co = NnState::kCh[k + 1];
        CK(nn_wgrad(q.G + q.off[k], q.part, gout, nn_act(ctx, k), ctx->U32, ctx->g, ci, co, 2.0 * gscale, ctx->st));
        if (k > 0) {
            CK(nn_layer(gin, gout, q.Wt[k], ctx->U32, ctx->g, co, ci, ctx->st));
            std::swap(gout, gin);
        }
    }
    return MG_OK;
}
int nn_need(mg_ctx* ctx) {
    TRY(need_links(ctx));
    if (!ctx->nn.weights) return fail(ctx, MG_ERR_NOT_SETUP, "no network weights: call mg_nn_set_weights");
    return MG_OK;
}
// n host random starts (boundary layout) -> x0 of start i in act
int nn_upload_start(mg_ctx* ctx, const double* eta_host, int i) {
    const size_t n = nfine(ctx);
    CK(cudaMemcpyAsync(ctx->stage_a, eta_host + 2 * (size_t)i * n, sizeof(double2) * n, cudaMemcpyHostToDevice, ctx->st));
    spinor_to_internal<float>((v2<float>*)nn_act(ctx, 0), ctx->stage_a, ctx->g, ctx->st);
    CKL();
    return MG_OK;
}
}  // namespace
extern "C" {

int mg_nn_set_weights(mg_ctx* ctx, const double* W, int ncomplex) {
    if (!ctx || !W) return MG_ERR_INVALID_ARG;
    if (ncomplex != kNnParams) return fail(ctx, MG_ERR_INVALID_ARG, "the network has 20736 complex weights");
    TRY(ensure_nn(ctx));
    CK(cudaMemcpyAsync(ctx->nn.Wm, W, sizeof(double2) * kNnParams, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemsetAsync(ctx->nn.m, 0, sizeof(double2) * kNnParams, ctx->st));
    CK(cudaMemsetAsync(ctx->nn.v, 0, sizeof(double2) * kNnParams, ctx->st));
    ctx->nn.step = 0;
    TRY(nn_refresh(ctx));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->nn.weights = true;
    return MG_OK;
}

int mg_nn_get_weights(mg_ctx* ctx, double* W, int ncomplex) {
    if (!ctx || !W) return MG_ERR_INVALID_ARG;
    if (ncomplex != kNnParams) return fail(ctx, MG_ERR_INVALID_ARG, "the network has 20736 complex weights");
    if (!ctx->nn.weights) return fail(ctx, MG_ERR_NOT_SETUP, "no network weights");
    CK(cudaMemcpyAsync(W, ctx->nn.Wm, sizeof(double2) * kNnParams, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

int mg_nn_forward(mg_ctx* ctx, const double* eta, double* v, int n) {
    if (!ctx || !eta || !v || n <= 0) return MG_ERR_INVALID_ARG;
    TRY(nn_need(ctx));
    const size_t nf = nfine(ctx);
    for (int i = 0; i < n; ++i) {
        TRY(nn_upload_start(ctx, eta, i));
        TRY(nn_forward(ctx));
        spinor_from_internal<float>(ctx->stage_b, (const v2<float>*)nn_act(ctx, NnState::kLayers), ctx->g, ctx->st);
        CKL();
        CK(cudaMemcpyAsync(v + 2 * (size_t)i * nf, ctx->stage_b, sizeof(double2) * nf, cudaMemcpyDeviceToHost, ctx->st));
    }
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

int mg_nn_loss_grad(mg_ctx* ctx, const double* eta, int n, double* loss, double* grad) {
    if (!ctx || !eta || n <= 0) return MG_ERR_INVALID_ARG;
    TRY(nn_need(ctx));
    TRY(need_level(ctx));
    CK(cudaMemsetAsync(ctx->nn.G, 0, sizeof(double2) * kNnParams, ctx->st));
    double tot = 0;
    for (int i = 0; i < n; ++i) {
        TRY(nn_upload_start(ctx, eta, i));
        TRY(nn_forward(ctx));
        TRY(nn_loss_grad(ctx, grad != nullptr, 1.0 / n));
        TRY(read_scalars(ctx, NN_V2, 2));
        tot += ctx->h_scal[NN_R2] / ctx->h_scal[NN_V2];
    }
    if (loss) *loss = tot / n;
    if (grad) {
        CK(cudaMemcpyAsync(grad, ctx->nn.G, sizeof(double2) * kNnParams, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    return MG_OK;
}

int mg_nn_train(mg_ctx* ctx, const double* eta, int n, int steps, double lr, double* loss_first, double* loss_last) {
    if (!ctx || !eta || n <= 0 || steps <= 0 || !(lr > 0)) return MG_ERR_INVALID_ARG;
    TRY(nn_need(ctx));
    TRY(need_level(ctx));
    NnState& q = ctx->nn;
    for (int it = 0; it < steps; ++it) {
        double l = 0;
        CK(cudaMemsetAsync(q.G, 0, sizeof(double2) * kNnParams, ctx->st));
        for (int i = 0; i < n; ++i) {
            TRY(nn_upload_start(ctx, eta, i));
            TRY(nn_forward(ctx));
            TRY(nn_loss_grad(ctx, true, 1.0 / n));
            TRY(read_scalars(ctx, NN_V2, 2));
            l += ctx->h_scal[NN_R2] / ctx->h_scal[NN_V2] / n;
        }
        q.step += 1;
        nn_adam(nullptr, q.Wm, q.G, q.m, q.v, kNnParams, lr, 0.9, 0.999, 1e-8, q.step, ctx->st);   // Adam on the FP64 weights
        TRY(nn_refresh(ctx));
        if (it == 0 && loss_first) *loss_first = l;
        if (loss_last) *loss_last = l;
    }
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

int mg_setup_learned(mg_ctx* ctx, const double* eta, int refine_iters) {
    if (!ctx || !eta || refine_iters < 0) return MG_ERR_INVALID_ARG;
    TRY(nn_need(ctx));
    TRY(ensure_protos(ctx));
    const size_t n = nfine(ctx);
    const int nv = ctx->prm.nvec;
    CK(cudaEventRecord(ctx->ev0, ctx->st));
    for (int i = 0; i < nv; ++i) {
        TRY(nn_upload_start(ctx, eta, i));
        TRY(nn_forward(ctx));
        convert<float, double>(ctx->protos + (size_t)i * n, (const v2<float>*)nn_act(ctx, NnState::kLayers), n,
                               ctx->st);
        norm2<double>(ctx->protos + (size_t)i * n, n, S_NORM_A, ctx->R, ctx->st);
        normalize_dev<double>(ctx->protos + (size_t)i * n, n, S_NORM_A, ctx->R, ctx->st);
    }
    CKL();
    const int iters = ctx->prm.setup_iters;
    ctx->prm.setup_iters = refine_iters;
    const int st = run_setup(ctx);
    ctx->prm.setup_iters = iters;
    return st;
}

// ---- the third level
}  // extern "C"
namespace {
int need_three_levels(mg_ctx* ctx) {
    if (ctx->prm.levels != 3) return fail(ctx, MG_ERR_INVALID_ARG, "the context was created with levels = 2");
    TRY(need_links(ctx));
    if (!ctx->full.valid) return fail(ctx, MG_ERR_NOT_SETUP, "no level-1 operator: run the fine setup first");
    return MG_OK;
}
int upload_protos2(mg_ctx* ctx, const double* V2) {
    const size_t n1 = (size_t)ctx->g.Vc * ctx->full.nc, nv2 = ctx->prm.nvec2;
    if (!ctx->protos2) {
        TRY(dalloc(ctx, &ctx->protos2, sizeof(double2) * n1 * nv2));
        TRY(dalloc(ctx, &ctx->protos2_t, sizeof(double2) * n1 * nv2));
    }
    CK(cudaMemcpyAsync(ctx->protos2, V2, sizeof(double2) * n1 * nv2, cudaMemcpyHostToDevice, ctx->st));
    return MG_OK;
}
template <typename T> int hook_kcycle(mg_ctx* ctx, const double* r1, double* e1) {
    TRY(ensure_work<T>(ctx));
    Work<T>& w = work<T>(ctx);
    const size_t n1 = (size_t)ctx->g.Vc * ctx->full.nc;
    CK(cudaMemcpyAsync(ctx->cstage, r1, sizeof(double2) * n1, cudaMemcpyHostToDevice, ctx->st));
    convert<double, T>(w.crc, ctx->cstage, n1, ctx->st);
    TRY(kcycle<T>(ctx, w.crc, w.cy));
    convert<T, double>(ctx->cstage, w.cy, n1, ctx->st);
    CKL();
    CK(cudaMemcpyAsync(e1, ctx->cstage, sizeof(double2) * n1, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return check_timeout(ctx);
}
}  // namespace
extern "C" {

int mg_setup_level2(mg_ctx* ctx, const double* V2) {
    if (!ctx || !V2) return MG_ERR_INVALID_ARG;
    TRY(need_three_levels(ctx));
    TRY(upload_protos2(ctx, V2));
    ctx->coarse16 = ctx->prm.prec_inner == MG_FP16;
    TRY(ctx->prm.prec_inner != MG_FP64 ? setup_level2_impl<float>(ctx) : setup_level2_impl<double>(ctx));
    return check_timeout(ctx);
}

int mg_set_level2_vectors(mg_ctx* ctx, const double* V2) {
    if (!ctx || !V2) return MG_ERR_INVALID_ARG;
    TRY(need_three_levels(ctx));
    TRY(upload_protos2(ctx, V2));
    return build_level2(ctx, ctx->full2, ctx->protos2, ctx->prm.nvec2);
}

int mg_get_level2_prolongator(mg_ctx* ctx, double* P2) {
    if (!ctx || !P2) return MG_ERR_INVALID_ARG;
    if (!ctx->full2.valid) return fail(ctx, MG_ERR_NOT_SETUP, "no level-2 prolongator");
    const CoarseLevel& L = ctx->full2;
    const int nv1 = ctx->prm.nvec, nv2 = L.nv, nc1 = 2 * nv1, vb = ctx->g2.Vb, len = vb * nv1;
    const size_t np = (size_t)nv2 * ctx->g.Vc * nc1;
    std::vector<double2> panel(np);
    CK(cudaMemcpyAsync(panel.data(), L.P64, sizeof(double2) * np, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    double2* out = reinterpret_cast<double2*>(P2);
    for (int X2 = 0; X2 < ctx->g2.Vc; ++X2)
        for (int sgn = 0; sgn < 2; ++sgn)
            for (int i = 0; i < nv2; ++i)
                for (int l2 = 0; l2 < vb; ++l2) {
                    const long long X1 = lex_site(ctx->g2, X2, l2);
                    for (int j = 0; j < nv1; ++j)
                        out[((size_t)i * ctx->g.Vc + X1) * nc1 + sgn * nv1 + j] =
                            panel[(((size_t)X2 * 2 + sgn) * nv2 + i) * len + (size_t)l2 * nv1 + j];
                }
    return MG_OK;
}

int mg_get_level2_op(mg_ctx* ctx, double* A2) {
    if (!ctx || !A2) return MG_ERR_INVALID_ARG;
    if (!ctx->full2.valid) return fail(ctx, MG_ERR_NOT_SETUP, "no level-2 operator");
    const CoarseLevel& L = ctx->full2;
    const size_t na = (size_t)ctx->g2.Vc * 9 * L.nc * L.nc;
    double2* tmp = nullptr;
    TRY(dalloc(ctx, &tmp, sizeof(double2) * na));
    coarse_op_transpose(tmp, L.A64, L.nc, ctx->g2.Vc, ctx->st);
    CKL();
    CK(cudaMemcpyAsync(A2, tmp, sizeof(double2) * na, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    dfree(ctx, tmp);
    return MG_OK;
}

int mg_kcycle(mg_ctx* ctx, const double* r1, double* e1, int prec) {
    if (!ctx || !r1 || !e1) return MG_ERR_INVALID_ARG;
    TRY(need_three_levels(ctx));
    if (!ctx->full2.valid) return fail(ctx, MG_ERR_NOT_SETUP, "no level-2 operator");
    ctx->coarse16 = prec == MG_FP16;
    return prec != MG_FP64 ? hook_kcycle<float>(ctx, r1, e1) : hook_kcycle<double>(ctx, r1, e1);
}

int mg_get_prolongator(mg_ctx* ctx, double* P) {
    TRY(need_level(ctx));
    if (!P) return MG_ERR_INVALID_ARG;
    size_t n = nfine(ctx);
    prolongator_to_boundary(ctx->protos_stage, ctx->full.P64, ctx->full.nv, ctx->g, ctx->st);
    CKL();
    CK(cudaMemcpyAsync(P, ctx->protos_stage, sizeof(double2) * n * ctx->full.nv, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

int mg_get_null_vectors(mg_ctx* ctx, double* V) {
    TRY(need_links(ctx));
    if (!V || !ctx->protos) return fail(ctx, MG_ERR_NOT_SETUP, "no prototypes");
    size_t n = nfine(ctx);
    for (int i = 0; i < ctx->prm.nvec; ++i)
        spinor_from_internal<double>(ctx->protos_stage + (size_t)i * n, ctx->protos + (size_t)i * n, ctx->g, ctx->st);
    CKL();
    CK(cudaMemcpyAsync(V, ctx->protos_stage, sizeof(double2) * n * ctx->prm.nvec, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

int mg_get_coarse_op(mg_ctx* ctx, double* A) {
    TRY(need_level(ctx));
    if (!A) return MG_ERR_INVALID_ARG;
    int nc = ctx->full.nc;
    coarse_op_transpose(ctx->cstage, ctx->full.A64, nc, ctx->g.Vc, ctx->st);
    CKL();
    CK(cudaMemcpyAsync(A, ctx->cstage, sizeof(double2) * (size_t)ctx->g.Vc * 9 * nc * nc, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

int mg_solve_device(mg_ctx* ctx, const double* b_dev, double* x_dev, mg_solve_info* info) {
    TRY(need_cycle(ctx));
    if (!b_dev || !x_dev) return fail(ctx, MG_ERR_INVALID_ARG, "null vector");
    spinor_to_internal<double>(ctx->b64, (const double2*)b_dev, ctx->g, ctx->st);
    CKL();
    ctx->coarse16 = ctx->prm.prec_inner == MG_FP16;
    int st = ctx->prm.prec_inner != MG_FP64 ? gcr_solve<float>(ctx, info) : gcr_solve<double>(ctx, info);
    if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return st;
    spinor_from_internal<double>((double2*)x_dev, ctx->x64, ctx->g, ctx->st);
    CKL();
    CK(cudaStreamSynchronize(ctx->st));
    return st;
}

int mg_solve(mg_ctx* ctx, const double* b, double* x, mg_solve_info* info) {
    TRY(need_cycle(ctx));
    if (!b || !x) return fail(ctx, MG_ERR_INVALID_ARG, "null vector");
    size_t n = nfine(ctx);
    CK(cudaMemcpyAsync(ctx->stage_a, b, sizeof(double2) * n, cudaMemcpyHostToDevice, ctx->st));
    int st = mg_solve_device(ctx, (const double*)ctx->stage_a, (double*)ctx->stage_b, info);
    if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return st;
    CK(cudaMemcpyAsync(x, ctx->stage_b, sizeof(double2) * n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return st;
}

int mg_apply_dslash(mg_ctx* ctx, const double* in, double* out, int prec) {
    TRY(need_links(ctx));
    if (!in || !out) return MG_ERR_INVALID_ARG;
    ctx->coarse16 = prec == MG_FP16;
    return prec != MG_FP64 ? hook_dslash<float>(ctx, in, out) : hook_dslash<double>(ctx, in, out);
}
int mg_restrict(mg_ctx* ctx, const double* r, double* rc, int prec) {
    TRY(need_level(ctx));
    if (!r || !rc) return MG_ERR_INVALID_ARG;
    ctx->coarse16 = prec == MG_FP16;
    return prec != MG_FP64 ? hook_restrict<float>(ctx, r, rc) : hook_restrict<double>(ctx, r, rc);
}
int mg_prolong(mg_ctx* ctx, const double* yc, double* e, int prec) {
    TRY(need_level(ctx));
    if (!yc || !e) return MG_ERR_INVALID_ARG;
    ctx->coarse16 = prec == MG_FP16;
    return prec != MG_FP64 ? hook_prolong<float>(ctx, yc, e) : hook_prolong<double>(ctx, yc, e);
}
int mg_apply_coarse(mg_ctx* ctx, const double* x, double* y, int dagger, int prec) {
    TRY(need_level(ctx));
    if (!x || !y) return MG_ERR_INVALID_ARG;
    ctx->coarse16 = prec == MG_FP16;
    return prec != MG_FP64 ? hook_coarse<float>(ctx, x, y, dagger) : hook_coarse<double>(ctx, x, y, dagger);
}
int mg_mr(mg_ctx* ctx, double* e, double* r, int nsteps, int prec) {
    TRY(need_links(ctx));
    if (!e || !r || nsteps < 0) return MG_ERR_INVALID_ARG;
    ctx->coarse16 = prec == MG_FP16;
    return prec != MG_FP64 ? hook_mr<float>(ctx, e, r, nsteps) : hook_mr<double>(ctx, e, r, nsteps);
}
int mg_coarse_solve(mg_ctx* ctx, const double* rc, double* y, double tol, int maxit, int prec, int* iters,
                    double* final_rel) {
    TRY(need_level(ctx));
    if (!rc || !y || maxit < 0) return MG_ERR_INVALID_ARG;
    ctx->coarse16 = prec == MG_FP16;
    return prec != MG_FP64 ? hook_coarse_solve<float>(ctx, rc, y, tol, maxit, iters, final_rel)
                           : hook_coarse_solve<double>(ctx, rc, y, tol, maxit, iters, final_rel);
}
int mg_vcycle(mg_ctx* ctx, const double* r, double* z, int prec) {
    TRY(need_cycle(ctx));
    if (!r || !z) return MG_ERR_INVALID_ARG;
    ctx->coarse16 = prec == MG_FP16;
    return prec != MG_FP64 ? hook_vcycle<float>(ctx, r, z) : hook_vcycle<double>(ctx, r, z);
}

// FP16-storage dslash for the timers: out = D in on the smoother's FP16 buffers
static int time_dslash_h(mg_ctx* ctx, int reps, void* flush, size_t flush_bytes, double* ms_per_launch) {
    TRY(ensure_work<float>(ctx));
    TRY(ensure_fine16(ctx));
    HalfSpinor a{ctx->h_r, ctx->h_sr}, b{ctx->h_q, ctx->h_sq};
    to_half(a, reinterpret_cast<const float2*>(work<float>(ctx).tin), ctx->g, ctx->st);
    for (int i = 0; i < 3; ++i) dslash_h_plain(b, a, ctx->U16, ctx->g, ctx->mass, ctx->st);
    double total = 0;
    if (!flush) CK(cudaEventRecord(ctx->ev0, ctx->st));
    for (int i = 0; i < reps; ++i) {
        if (flush) {
            CK(cudaMemsetAsync(flush, i & 0xff, flush_bytes, ctx->st));
            CK(cudaEventRecord(ctx->ev0, ctx->st));
        }
        dslash_h_plain(b, a, ctx->U16, ctx->g, ctx->mass, ctx->st);
        if (flush) {
            CK(cudaEventRecord(ctx->ev1, ctx->st));
            CK(cudaEventSynchronize(ctx->ev1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
            total += ms;
        }
    }
    if (!flush) {
        CK(cudaEventRecord(ctx->ev1, ctx->st));
        CK(cudaEventSynchronize(ctx->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        total = ms;
    }
    CKL();
    *ms_per_launch = total / reps;
    return MG_OK;
}

int mg_time_dslash(mg_ctx* ctx, int prec, int reps, double* ms_per_launch, double* bytes_per_launch) {
    TRY(need_links(ctx));
    if (reps <= 0 || !ms_per_launch) return MG_ERR_INVALID_ARG;
    if (prec == MG_FP16) {
        // links 4 x 5 pair words + input and output 12 half2 + one FP32 scale each per site
        if (bytes_per_launch) *bytes_per_launch = (double)ctx->g.V * (160 + 52 + 52);
        return time_dslash_h(ctx, reps, nullptr, 0, ms_per_launch);
    }
    size_t real = prec != MG_FP64 ? 4 : 8;
    // algorithmic minimum: 4 links x 18 reals + input 24 reals + output 24 reals per site
    if (bytes_per_launch) *bytes_per_launch = (double)ctx->g.V * (72 + 24 + 24) * real;
    auto run = [&](auto tag) -> int {
        using T = decltype(tag);
        TRY(ensure_work<T>(ctx));
        Work<T>& w = work<T>(ctx);
        const v2<T>* U = links<T>(ctx);
        for (int i = 0; i < 3; ++i)
            dslash<T>(DS_PLAIN, w.tout, w.tin, U, w.tin, ctx->g, ctx->mass, 0.0, 0, ctx->R, ctx->st);
        CK(cudaEventRecord(ctx->ev0, ctx->st));
        for (int i = 0; i < reps; ++i)   // same input every time (no growth to overflow)
            dslash<T>(DS_PLAIN, w.tout, w.tin, U, w.tin, ctx->g, ctx->mass, 0.0, 0, ctx->R, ctx->st);
        CK(cudaEventRecord(ctx->ev1, ctx->st));
        CKL();
        CK(cudaEventSynchronize(ctx->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        *ms_per_launch = ms / reps;
        return MG_OK;
    };
    return prec != MG_FP64 ? run(float{}) : run(double{});
}

int mg_time_coarse_floor(mg_ctx* ctx, int rounds, double* us_stencils, double* us_exchange) {
    TRY(need_level(ctx));
    if (rounds <= 0 || !us_stencils || !us_exchange) return MG_ERR_INVALID_ARG;
    if (ctx->prm.prec_inner == MG_FP64 || ctx->prm.coarse_kernel == 1)
        return fail(ctx, MG_ERR_INVALID_ARG, "the latency probes run the on-chip coarse solver (FP32 or FP16 inner precision)");
    TRY(ensure_work<float>(ctx));
    CoarseLevel& L = ctx->full;
    const CgSys<float> sys = level1_sys<float>(ctx);
    const int mode = cgls_mode(ctx->prm.coarse_kernel);
    bool onchip = false;
    TRY(ensure_units(ctx, L, sys.g.Vc, ctx->coarse16, mode, &onchip));
    if (!onchip) return fail(ctx, MG_ERR_INVALID_ARG, "no on-chip shape for this coarse level");
    double* outs[2] = {us_stencils, us_exchange};
    const int forms[2] = {CGLS_PROBE_STENCILS, CGLS_PROBE_EXCHANGE};
    for (int f = 0; f < 2; ++f) {
        CglsArgs c{};
        c.Au = L.Au; c.su = ctx->coarse16 ? L.su : nullptr; c.nbr = sys.nbr;
        c.rc = (const float2*)sys.cr; c.y = (float2*)sys.cp; c.r = (float2*)sys.cr1; c.r1 = (float2*)sys.cr1;
        c.s = (float2*)sys.cs; c.p = (float2*)sys.cp; c.p1 = (float2*)sys.cp1; c.q = (float2*)sys.cq;
        c.nc = L.nc; c.g = sys.g; c.tol2 = 0.f; c.maxit = rounds;
        c.scal = ctx->scal_s; c.err = (int*)(ctx->bar + 2);
        c.sh = L.au_shape;
        const unsigned long long reserve = 2ull * (unsigned long long)rounds + 4ull;
        if ((unsigned long long)ctx->xch_epoch + reserve >= 0xFFFFFFFFull) {
            CK(cudaMemsetAsync(ctx->xch, 0, sizeof(unsigned long long) * kXchWords, ctx->st));
            TRY(clear_epoch_tags(ctx));
            ctx->xch_epoch = 1;
        }
        c.xch = ctx->xch;
        c.epoch0 = ctx->xch_epoch;
        c.form = forms[f];
        c.tag = sys.ctag;
        ctx->xch_epoch += (unsigned int)reserve;
        CK(cudaMemsetAsync(ctx->bar, 0, sizeof(unsigned int) * 3, ctx->st));
        CK(cudaEventRecord(ctx->ev0, ctx->st));
        CK(cgls_onchip(c, ctx->st));
        CK(cudaEventRecord(ctx->ev1, ctx->st));
        CK(cudaEventSynchronize(ctx->ev1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        TRY(check_timeout(ctx));
        *outs[f] = 1e3 * (double)ms / rounds;
    }
    return MG_OK;
}

int mg_time_dslash_cold(mg_ctx* ctx, int prec, int reps, void* flush, size_t flush_bytes, double* ms_per_launch,
                        double* bytes_per_launch) {
    TRY(need_links(ctx));
    if (reps <= 0 || !ms_per_launch || !flush || flush_bytes == 0) return MG_ERR_INVALID_ARG;
    if (prec == MG_FP16) {
        if (bytes_per_launch) *bytes_per_launch = (double)ctx->g.V * (160 + 52 + 52);
        return time_dslash_h(ctx, reps, flush, flush_bytes, ms_per_launch);
    }
    size_t real = prec != MG_FP64 ? 4 : 8;
    if (bytes_per_launch) *bytes_per_launch = (double)ctx->g.V * (72 + 24 + 24) * real;
    auto run = [&](auto tag) -> int {
        using T = decltype(tag);
        TRY(ensure_work<T>(ctx));
        Work<T>& w = work<T>(ctx);
        const v2<T>* U = links<T>(ctx);
        for (int i = 0; i < 3; ++i)
            dslash<T>(DS_PLAIN, w.tout, w.tin, U, w.tin, ctx->g, ctx->mass, 0.0, 0, ctx->R, ctx->st);
        double total = 0;
        for (int i = 0; i < reps; ++i) {
            // overwrite a buffer larger than L2 so that links and spinors come from HBM
            CK(cudaMemsetAsync(flush, i & 0xff, flush_bytes, ctx->st));
            CK(cudaEventRecord(ctx->ev0, ctx->st));
            dslash<T>(DS_PLAIN, w.tout, w.tin, U, w.tin, ctx->g, ctx->mass, 0.0, 0, ctx->R, ctx->st);
            CK(cudaEventRecord(ctx->ev1, ctx->st));
            CKL();
            CK(cudaEventSynchronize(ctx->ev1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
            total += ms;
        }
        *ms_per_launch = total / reps;
        return MG_OK;
    };
    return prec != MG_FP64 ? run(float{}) : run(double{});
}

int mg_profile_enable(mg_ctx* ctx, int on) {
    if (!ctx) return MG_ERR_INVALID_ARG;
    ctx->prof = on != 0;
    return MG_OK;
}

int mg_profile_classes(mg_ctx* ctx, unsigned int mask) {
    if (!ctx) return MG_ERR_INVALID_ARG;
    if (!(mask & ((1u << MG_K_NCLASSES) - 1u))) return fail(ctx, MG_ERR_INVALID_ARG, "the mask selects no kernel class");
    if (!ctx->ev_class.empty()) return fail(ctx, MG_ERR_INVALID_ARG, "read the launch timer before changing its classes");
    ctx->prof_mask = mask;
    return MG_OK;
}

int mg_profile_read(mg_ctx* ctx, double* ms, int* launches, double* coarse_iters) {
    if (!ctx || !ms || !launches) return MG_ERR_INVALID_ARG;
    for (int c = 0; c < MG_K_NCLASSES; ++c) { ms[c] = 0.0; launches[c] = 0; }
    TRY(read_scalars(ctx, S_CG_TOTAL, 1));
    if (coarse_iters) *coarse_iters = ctx->h_scal[S_CG_TOTAL] - ctx->coarse_mark;
    ctx->coarse_mark = ctx->h_scal[S_CG_TOTAL];
    for (size_t i = 0; i < ctx->ev_class.size(); ++i) {
        float t = 0;
        CK(cudaEventElapsedTime(&t, ctx->ev_pool[2 * i], ctx->ev_pool[2 * i + 1]));
        ms[ctx->ev_class[i]] += t;
        launches[ctx->ev_class[i]] += 1;
    }
    ctx->ev_class.clear();
    ctx->ev_used = 0;
    return MG_OK;
}

long long mg_kernel_launches(void) { return launch_counter().load(std::memory_order_relaxed); }

int mg_check_wait_timeout(mg_ctx* ctx, int kind, long long spin_limit) {
    if (!ctx) return MG_ERR_INVALID_ARG;
    if (kind < 0 || kind > 3 || spin_limit < 1 || spin_limit > 10000000LL)
        return fail(ctx, MG_ERR_INVALID_ARG, "kind must be 0..3 and spin_limit in 1..1e7");
    const int G = 4;
    const size_t words = (size_t)2 * 3 * (G + 1) * 16;   // two parities x three values x (G + 1) padded slots
    unsigned long long* w = nullptr;
    unsigned int* ctr = nullptr;
    TRY(dalloc(ctx, &w, sizeof(unsigned long long) * words));
    TRY(dalloc(ctx, &ctr, sizeof(unsigned int) * 4));   // [0] count, [1] generation, [2] error flag
    int st = MG_OK;
    CK(cudaMemsetAsync(w, 0, sizeof(unsigned long long) * words, ctx->st));
    CK(cudaMemsetAsync(ctr, 0, sizeof(unsigned int) * 4, ctx->st));
    CK(wait_probe(kind, G, w, ctr, (int*)(ctr + 2), spin_limit, ctx->st));
    unsigned int flag = 0;
    CK(cudaMemcpyAsync(&flag, ctr + 2, sizeof(flag), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    dfree(ctx, w);
    dfree(ctx, ctr);
    if (flag) st = fail(ctx, MG_ERR_TIMEOUT, "bounded wait gave up as expected (kind " + std::to_string(kind) + ")");
    return st;
}
int mg_coarse_kernel(mg_ctx* ctx) { return ctx ? ctx->coarse_kernel_used : MG_CK_NONE; }

const char* mg_status_string(int status) {
    int i = -status;
    if (i < 0 || i >= (int)(sizeof(kStatusNames) / sizeof(kStatusNames[0]))) return "MG_ERR_UNKNOWN";
    return kStatusNames[i];
}

const char* mg_last_error(const mg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

}  // extern "C"

// ======================================================================= allocation-free coarse solve
// For callers that must not allocate device memory at call time: code running
// while another framework owns the device allocator, or work issued from a
// context where cudaMalloc is not allowed or would synchronise the device
// (a real-time loop, a host callback, code between a setup done at start-up
// and the end of the program).  The CG work vectors, the reduction partial
// sums, the arrival counter and the solver scalars live in one file-scope
// __device__ array instead of context memory.  Every GPU that loads this
// library holds the array until the process exits.
namespace {

constexpr size_t kNoAllocMaxCoarseDof = 65536;              // coarse sites x 2 Nv
constexpr size_t kNoAllocVecBytes = kNoAllocMaxCoarseDof * sizeof(double2);
constexpr size_t kNoAllocPartialsBytes = (size_t)kMaxReduceBlocks * 64 * sizeof(double);
constexpr size_t kNoAllocScalBytes = ((S_COUNT * sizeof(double) + 255) / 256) * 256;
constexpr size_t kNoAllocScratchBytes = 6 * kNoAllocVecBytes + kNoAllocPartialsBytes + kNoAllocScalBytes + 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the lookup also loads the module on that device).
int noalloc_scratch(mg_ctx* ctx, unsigned char** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev != ctx->dev)
        return fail(ctx, MG_ERR_INVALID_ARG,
                    "the current device (" + std::to_string(dev) + ") is not the context's device (" +
                        std::to_string(ctx->dev) + "): make the context's device current before this call");
    if (dev < 0 || dev >= kMaxDevices) return fail(ctx, MG_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(ctx, MG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = (unsigned char*)p;
    }
    *out = g_noalloc_addr[dev];
    return MG_OK;
}

}  // namespace

extern "C" int mg_coarse_solve_noalloc(mg_ctx* ctx, const double* rc_dev, double* y_dev, double tol, int maxit,
                                       int* iters, double* final_rel) {
    TRY(need_level(ctx));
    if (!rc_dev || !y_dev || maxit < 0) return fail(ctx, MG_ERR_INVALID_ARG, "null buffer or negative maxit");
    const CoarseLevel& L = ctx->full;
    size_t n = (size_t)ctx->g.Vc * L.nc;
    if (n > kNoAllocMaxCoarseDof)
        return fail(ctx, MG_ERR_INVALID_ARG,
                    "coarse vector of " + std::to_string(n) + " complex entries exceeds the allocation-free limit of " +
                        std::to_string(kNoAllocMaxCoarseDof));
    unsigned char* base = nullptr;
    TRY(noalloc_scratch(ctx, &base));
    v2<double>* r = (v2<double>*)base;
    v2<double>* r1 = (v2<double>*)(base + kNoAllocVecBytes);
    v2<double>* s = (v2<double>*)(base + 2 * kNoAllocVecBytes);
    v2<double>* p = (v2<double>*)(base + 3 * kNoAllocVecBytes);
    v2<double>* p1 = (v2<double>*)(base + 4 * kNoAllocVecBytes);
    v2<double>* q = (v2<double>*)(base + 5 * kNoAllocVecBytes);
    Reduce R;
    R.partials = (double*)(base + 6 * kNoAllocVecBytes);
    R.scal = (double*)(base + 6 * kNoAllocVecBytes + kNoAllocPartialsBytes);
    R.ticket = (unsigned int*)(base + 6 * kNoAllocVecBytes + kNoAllocPartialsBytes + kNoAllocScalBytes);
    R.partial_bytes = kNoAllocPartialsBytes;
    // the barrier counters and the error flag must start at zero; everything
    // else is written before it is read
    unsigned int* bar = R.ticket;
    CK(cudaMemsetAsync(bar, 0, sizeof(unsigned int) * 3, ctx->st));
    CgnrArgs<double> a = cgnr_args<double>(L, ctx->g, (const v2<double>*)rc_dev, (v2<double>*)y_dev, r, r1, s, p, p1, q,
                                           tol, maxit, R.partials, bar, R.scal);
    a.nbr = ctx->cnbr;   // context memory made at create (an input, not an allocation here)
    CK(cgnr_persistent<double>(a, ctx->st));
    CK(cudaMemcpyAsync(ctx->h_scal + S_CG_RC2, R.scal + S_CG_RC2, sizeof(double) * 3, cudaMemcpyDeviceToHost, ctx->st));
    unsigned int flags[3];
    CK(cudaMemcpyAsync(flags, bar, sizeof(flags), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (flags[2]) return fail(ctx, MG_ERR_TIMEOUT, "coarse solve: a grid barrier wait gave up");
    if (iters) *iters = (int)ctx->h_scal[S_CG_ITERS];
    if (final_rel)
        *final_rel = ctx->h_scal[S_CG_RC2] > 0 ? std::sqrt(ctx->h_scal[S_CG_R2] / ctx->h_scal[S_CG_RC2]) : 0.0;
    return MG_OK;
}

// ======================================================================= red-black preconditioned CG
// The comparison solver of Sec. IV: CG on the normal equations of the
// even-site Schur complement Dhat = (4+m) - H_eo H_oe / (4+m), inner
// iterations in T (FP32 or FP64) with the solution accumulated in FP64; each
// cycle restarts the CG on the FP64 true residual (defect correction) until
// ||b - D x|| <= tol ||b||.
namespace {

constexpr int kEoCheck = 16;   // CG iterations queued between host reads of the done flag
constexpr double kEoInnerDelta = 0.1;    // FP32 inner solve: residual reduction between reliable updates

int ensure_eo(mg_ctx* ctx, int inner_bytes) {
    EoWork& w = ctx->eo;
    const Geom& g = ctx->g;
    if (!w.U64) {
        for (int mu = 0; mu < 4; ++mu)
            if (g.L[mu] % 2) return fail(ctx, MG_ERR_INVALID_ARG, "red-black CG needs even lattice extents");
        w.e.Lh0 = g.L[0] / 2;
        for (int mu = 0; mu < 4; ++mu) w.e.L[mu] = g.L[mu];
        w.e.Vh = g.V / 2;
        w.e.tap = g.tap;
        const size_t nf = (size_t)24 * w.e.Vh;
        TRY(dalloc(ctx, &w.U64, sizeof(double2) * 36 * (size_t)g.V));
        TRY(dalloc(ctx, &w.U32, sizeof(float2) * 36 * (size_t)g.V));
        TRY(dalloc(ctx, &w.b, sizeof(double2) * nf));
        TRY(dalloc(ctx, &w.x, sizeof(double2) * nf));
        TRY(dalloc(ctx, &w.res, sizeof(double2) * nf));
        TRY(dalloc(ctx, &w.t, sizeof(double2) * nf));
    }
    if (w.inner_bytes != inner_bytes) {
        for (void* q : {w.xe, w.r, w.s, w.p, w.q, w.t1}) dfree(ctx, q);
        const size_t nh = (size_t)12 * w.e.Vh * inner_bytes;
        for (void** q : {&w.xe, &w.r, &w.s, &w.p, &w.q, &w.t1}) {
            unsigned char* a = nullptr;
            TRY(dalloc(ctx, &a, nh));
            *q = a;
        }
        w.inner_bytes = inner_bytes;
    }
    if (!w.links_valid) {
        eo_links_pack(w.U64, w.U32, ctx->U64, g, w.e, ctx->st);
        CKL();
        w.links_valid = true;
    }
    return MG_OK;
}

// b_dev, x_dev: boundary-layout FP64 device spinors
template <typename T>
int eo_cg_solve(mg_ctx* ctx, const double2* b_dev, double2* x_dev, double tol, int maxit, mg_solve_info* info) {
    TRY(need_links(ctx));
    if (!(tol > 0) || maxit < 0) return fail(ctx, MG_ERR_INVALID_ARG, "tol must be > 0 and maxit >= 0");
    TRY(ensure_eo(ctx, (int)sizeof(v2<T>)));
    EoWork& w = ctx->eo;
    const EoGeom& e = w.e;
    const Reduce& R = ctx->R;
    const long long nh = 12 * e.Vh;
    const double a = 4.0 + ctx->mass, ainv = 1.0 / a;
    const void* Ui = sizeof(T) == 4 ? (const void*)w.U32 : (const void*)w.U64;
    v2<T>*xe = (v2<T>*)w.xe, *r = (v2<T>*)w.r, *sv = (v2<T>*)w.s, *p = (v2<T>*)w.p, *q = (v2<T>*)w.q,
         *t1 = (v2<T>*)w.t1;
    double2 *be = w.b, *bo = w.b + nh, *xe64 = w.x, *xo64 = w.x + nh, *re = w.res, *ro = w.res + nh;
    double2 *te = w.t, *to = w.t + nh;
    enum { G0 = S_EO, G1 = S_EO + 1, Q2 = S_EO + 2, R2 = S_EO + 3, TOL2 = S_EO + 4, DONE = S_EO + 5, ITS = S_EO + 6,
           RE2 = S_EO + 7, RO2 = S_EO + 8, B2 = S_EO + 9 };
    long long half_hops = 0, products = 0;   // half-lattice hops (bytes); matrix products (the count of Fig. 1)
    int iters = 0, cycles = 0, status = MG_ERR_NOT_CONVERGED;
    CK(cudaEventRecord(ctx->ev0, ctx->st));
    eo_spinor_pack<double>(w.b, b_dev, e, ctx->st);
    zero<double>(w.x, 2 * nh, ctx->st);
    CK(cudaMemcpyAsync(w.res, w.b, sizeof(double2) * 2 * nh, cudaMemcpyDeviceToDevice, ctx->st));
    norm2<double>(w.b, 2 * nh, B2, R, ctx->st);
    CKL();
    TRY(read_scalars(ctx, B2, 1));
    const double bnorm = std::sqrt(ctx->h_scal[B2]);
    ctx->h_scal[ITS] = 0.0;
    CK(cudaMemcpyAsync(R.scal + ITS, ctx->h_scal + ITS, sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    double rel = bnorm > 0 ? 1.0 : 0.0, rnorm = bnorm;
    if (!std::isfinite(bnorm)) return fail(ctx, MG_ERR_NUMERIC, "right-hand side is not finite");
    if (bnorm == 0) status = MG_OK;
    const double delta = sizeof(T) == 4 ? kEoInnerDelta : 0.0;
    // Reliable updates: every cycle ends with the FP64 residual of the
    // accumulated solution; the next cycle replaces the CG residual by it and
    // keeps the search direction (p = D^dag r + beta p with beta from the new
    // |D^dag r|^2), so the FP32 iterations continue one CG instead of
    // restarting it.  jg is the global iteration index: gamma_j = |s_j|^2
    // lives in slot G0 + (j & 1).
    int jg = 0;
    while (status == MG_ERR_NOT_CONVERGED && iters < maxit) {
        // bhat = res_e + H_eo res_o / (4+m) -> the inner right-hand side r, x_e = 0
        eo_hop<double>(EO_SRC, te, ro, re, nullptr, w.U64, e, 0, 1.0, 0.0, ainv, 0, DONE, R, ctx->st);
        half_hops += 1;
        convert<double, T>(r, te, nh, ctx->st);
        zero<T>(xe, nh, ctx->st);
        // the inner residual equals b - D x in exact arithmetic; a drift is
        // caught by the FP64 residual at the end of the cycle
        const double target = std::max(delta * rnorm, tol * bnorm);
        ctx->h_scal[TOL2] = target * target;
        ctx->h_scal[DONE] = 0.0;
        CK(cudaMemcpyAsync(R.scal + TOL2, ctx->h_scal + TOL2, sizeof(double) * 2, cudaMemcpyHostToDevice, ctx->st));
        // s = Dhat^dag r = (4+m) r - gamma5 H_eo H_oe gamma5 r / (4+m); gamma_jg = |s|^2
        const int gj = (jg & 1) ? G1 : G0, gprev = (jg & 1) ? G0 : G1;
        eo_hop<T>(EO_G5IN, t1, r, nullptr, nullptr, Ui, e, 1, 0.0, 0.0, 1.0, 0, DONE, R, ctx->st);
        eo_hop<T>(EO_SELF | EO_NORM | EO_G5H, sv, t1, nullptr, r, Ui, e, 0, 0.0, a, -ainv, gj, DONE, R, ctx->st);
        half_hops += 2;
        if (jg == 0) CK(cudaMemcpyAsync(p, sv, sizeof(v2<T>) * nh, cudaMemcpyDeviceToDevice, ctx->st));
        else eo_cg_update2<T>(p, sv, nh, gprev, gj, DONE, R, ctx->st);
        CKL();
        const int budget = maxit - iters;
        int queued = 0, done_its = 0;
        for (;;) {
            const int n = std::min(kEoCheck, budget - queued);
            for (int j = jg + queued; j < jg + queued + n; ++j) {
                const int g_old = (j & 1) ? G1 : G0, g_new = (j & 1) ? G0 : G1;
                EoCgSlots sl{g_old, Q2, R2, TOL2, DONE, ITS};
                // q = Dhat p, |q|^2
                eo_hop<T>(EO_SKIP, t1, p, nullptr, nullptr, Ui, e, 1, 0.0, 0.0, 1.0, 0, DONE, R, ctx->st);
                eo_hop<T>(EO_SKIP | EO_SELF | EO_NORM, q, t1, nullptr, p, Ui, e, 0, 0.0, a, -ainv, Q2, DONE, R, ctx->st);
                // x_e += alpha p, r -= alpha q, |r|^2, convergence
                eo_cg_update1<T>(xe, r, p, q, nh, sl, j, R, ctx->st);
                // s = Dhat^dag r, |s|^2 -> the new gamma; p = s + beta p
                eo_hop<T>(EO_SKIP | EO_G5IN, t1, r, nullptr, nullptr, Ui, e, 1, 0.0, 0.0, 1.0, 0, DONE, R, ctx->st);
                eo_hop<T>(EO_SKIP | EO_SELF | EO_NORM | EO_G5H, sv, t1, nullptr, r, Ui, e, 0, 0.0, a, -ainv, g_new, DONE,
                          R, ctx->st);
                eo_cg_update2<T>(p, sv, nh, g_old, g_new, DONE, R, ctx->st);
            }
            CKL();
            queued += n;
            TRY(read_scalars(ctx, DONE, 2));
            done_its = (int)ctx->h_scal[ITS] - jg;
            if (ctx->h_scal[DONE] != 0.0 || queued >= budget) break;
        }
        // the last iteration's D^dag r is skipped once the CG has stopped
        const int skipped = done_its > 0 && ctx->h_scal[DONE] != 0.0 ? 1 : 0;
        iters += done_its;
        jg += done_its;
        half_hops += 4LL * done_its - 2 * skipped;
        // per cycle: bhat, Dhat^dag r_0, Dhat and Dhat^dag per iteration, x_o, the residual
        products += 1 + 1 + 2LL * done_its - skipped + 1 + 1;
        // x_e += x_e(inner); x_o += (res_o + H_oe x_e(inner)) / (4+m), in FP64
        convert<T, double>(te, xe, nh, ctx->st);
        axpy<double>(xe64, te, nh, 1.0, 0.0, ctx->st);
        eo_hop<double>(EO_SRC | EO_ACC, xo64, te, ro, nullptr, w.U64, e, 1, ainv, 0.0, ainv, 0, DONE, R, ctx->st);
        // the true residual b - D x in FP64 on both parities
        eo_hop<double>(EO_SRC | EO_SELF | EO_NORM, re, xo64, be, xe64, w.U64, e, 0, 1.0, -a, 1.0, RE2, DONE, R, ctx->st);
        eo_hop<double>(EO_SRC | EO_SELF | EO_NORM, ro, xe64, bo, xo64, w.U64, e, 1, 1.0, -a, 1.0, RO2, DONE, R, ctx->st);
        half_hops += 3;
        CKL();
        TRY(read_scalars(ctx, RE2, 2));
        ++cycles;
        rnorm = std::sqrt(ctx->h_scal[RE2] + ctx->h_scal[RO2]);
        rel = rnorm / bnorm;
        if (!std::isfinite(rel)) { status = MG_ERR_NUMERIC; break; }
        if (rel <= tol) status = MG_OK;
        else if (done_its == 0) { status = MG_ERR_NUMERIC; break; }   // no progress possible
    }
    eo_spinor_unpack<double>(x_dev, w.x, e, ctx->st);
    CKL();
    CK(cudaEventRecord(ctx->ev1, ctx->st));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (info) {
        info->outer_iters = iters;
        info->coarse_iters = 0;
        info->fine_matvecs = (int)products;
        info->restarts = cycles;
        info->true_rel_res = rel;
        info->solve_ms = ms;
        info->status = status;
        info->setup_ms = 0.0;
        // per half-lattice hop: all 4 V links once, the input and output half vectors
        const double per_site = sizeof(T) == 4 ? (288.0 + 96.0) : (576.0 + 192.0);
        info->dslash_bytes = (double)half_hops * per_site * (double)ctx->g.V;
    }
    if (status == MG_ERR_NOT_CONVERGED) ctx->err = "red-black CG: maxit reached";
    if (status == MG_ERR_NUMERIC) ctx->err = "red-black CG: non-finite residual or no progress";
    return status;
}

}  // namespace

extern "C" int mg_solve_eo_cg_device(mg_ctx* ctx, const double* b_dev, double* x_dev, double tol, int maxit, int prec,
                                     mg_solve_info* info) {
    if (!ctx || !b_dev || !x_dev) return MG_ERR_INVALID_ARG;
    if (prec != MG_FP64 && prec != MG_FP32) return fail(ctx, MG_ERR_INVALID_ARG, "prec must be MG_FP64 or MG_FP32");
    int st = prec == MG_FP64 ? eo_cg_solve<double>(ctx, (const double2*)b_dev, (double2*)x_dev, tol, maxit, info)
                             : eo_cg_solve<float>(ctx, (const double2*)b_dev, (double2*)x_dev, tol, maxit, info);
    if (st == MG_OK || st == MG_ERR_NOT_CONVERGED) CK(cudaStreamSynchronize(ctx->st));
    return st;
}

extern "C" int mg_solve_eo_cg(mg_ctx* ctx, const double* b, double* x, double tol, int maxit, int prec,
                              mg_solve_info* info) {
    if (!ctx || !b || !x) return MG_ERR_INVALID_ARG;
    const size_t n = nfine(ctx);
    CK(cudaMemcpyAsync(ctx->stage_a, b, sizeof(double2) * n, cudaMemcpyHostToDevice, ctx->st));
    int st = mg_solve_eo_cg_device(ctx, (const double*)ctx->stage_a, (double*)ctx->stage_b, tol, maxit, prec, info);
    if (st == MG_OK || st == MG_ERR_NOT_CONVERGED) {
        CK(cudaMemcpyAsync(x, ctx->stage_b, sizeof(double2) * n, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    return st;
}

// ======================================================================= batched right-hand sides
// Lockstep flexible GCR over nrhs sources: the fine-level steps of each source
// use the single-source kernels, the coarse solve of all sources runs as one
// batched CGNR on an RHS panel (tensor-core stencil, iterations replayed from a
// captured CUDA graph), each source keeps its own GCR scalars.
namespace {

constexpr int kBatchCheck = 8;   // coarse iterations per graph replay between host checks

int round16(int n) { return ((n + 15) / 16) * 16; }

int ensure_embedding(mg_ctx* ctx, CoarseLevel& L) {
    if (L.emb_valid) return MG_OK;
    // per (X, d) block: the (2 nc) x (2 nc) real embedding, nc = 2 nv
    const size_t kemb = (size_t)4 * L.cap;
    if (!L.Aemb) TRY(dalloc(ctx, &L.Aemb, sizeof(__half) * (size_t)ctx->g.Vc * 9 * kemb * kemb));
    coarse_embed(L.Aemb, L.A64, L.nc, ctx->g.Vc, ctx->st);
    CKL();
    L.emb_valid = true;
    return MG_OK;
}

int ensure_batch(mg_ctx* ctx, int nrhs) {
    BatchWork& b = ctx->bw;
    int npad = round16(nrhs), nc = ctx->full.nc;
    size_t n = nfine(ctx);
    int K = std::min(ctx->prm.gcr_restart, ctx->K);
    if (b.npad >= npad && b.nrhs_cap >= nrhs && b.nc == nc && b.K >= K) return MG_OK;
    if (b.npad || b.nrhs_cap) {   // grow: release the smaller workspace first
        CK(cudaStreamSynchronize(ctx->st));
        for (void* q : {(void*)b.rcB, (void*)b.yB, (void*)b.rB, (void*)b.sB, (void*)b.pB, (void*)b.qB, (void*)b.cgs,
                        (void*)b.bt,
                        (void*)b.xpart, (void*)b.rpart, (void*)b.flags, (void*)b.r32, (void*)b.Z, (void*)b.Pk,
                        (void*)b.x64, (void*)b.b64, (void*)b.scal})
            dfree(ctx, q);
        if (b.graph) cudaGraphExecDestroy(b.graph);
        if (b.cap) cudaStreamDestroy(b.cap);
        cudaFreeHost(b.h_flags);
        cudaFreeHost(b.h_iters);
        cudaFreeHost(b.h_scal);
        b = BatchWork{};
        npad = std::max(npad, round16(nrhs));
    }
    size_t pe = (size_t)ctx->g.Vc * nc * npad;
    TRY(dalloc(ctx, &b.rcB, sizeof(float2) * pe));
    TRY(dalloc(ctx, &b.yB, sizeof(float2) * pe));
    TRY(dalloc(ctx, &b.rB, sizeof(float2) * pe));
    TRY(dalloc(ctx, &b.sB, sizeof(float2) * pe));
    TRY(dalloc(ctx, &b.pB, sizeof(float2) * pe));
    TRY(dalloc(ctx, &b.qB, sizeof(float2) * pe));
    TRY(dalloc(ctx, &b.cgs, sizeof(double) * 9 * npad));
    TRY(dalloc(ctx, &b.bt, tc_split_bytes(nc, npad, ctx->g.Vc)));
    TRY(dalloc(ctx, &b.xpart, sizeof(float) * (size_t)ctx->g.Vc * npad));
    TRY(dalloc(ctx, &b.rpart, sizeof(float) * kBatchRowChunks * npad));
    TRY(dalloc(ctx, &b.flags, sizeof(int) * 4));
    TRY(dalloc(ctx, &b.r32, sizeof(float2) * n * nrhs));
    TRY(dalloc(ctx, &b.Z, sizeof(float2) * n * nrhs * K));
    TRY(dalloc(ctx, &b.Pk, sizeof(float2) * n * nrhs * K));
    TRY(dalloc(ctx, &b.x64, sizeof(double2) * n * nrhs));
    TRY(dalloc(ctx, &b.b64, sizeof(double2) * n * nrhs));
    TRY(dalloc(ctx, &b.scal, sizeof(double) * S_COUNT * nrhs));
    CK(cudaMallocHost(&b.h_flags, sizeof(int) * 4));
    CK(cudaMallocHost(&b.h_iters, sizeof(double) * npad));
    CK(cudaMallocHost(&b.h_scal, sizeof(double) * S_COUNT * nrhs));
    CK(cudaStreamCreateWithFlags(&b.cap, cudaStreamNonBlocking));
    CK(cudaMemsetAsync(b.scal, 0, sizeof(double) * S_COUNT * nrhs, ctx->st));
    CK(cudaMemsetAsync(b.flags, 0, sizeof(int) * 4, ctx->st));
    b.npad = npad;
    b.nrhs_cap = nrhs;
    b.nc = nc;
    b.K = K;
    return MG_OK;
}

BatchCg batch_cg(mg_ctx* ctx, double tol, int maxit, int nrhs) {
    BatchWork& b = ctx->bw;
    BatchCg c;
    c.Aemb = ctx->full.Aemb;
    c.bt = b.bt;
    c.stages = 0;
    c.y = b.yB; c.r = b.rB; c.s = b.sB; c.p = b.pB; c.q = b.qB; c.rc = b.rcB;
    c.nc = ctx->full.nc; c.npad = b.npad; c.nw = b.npad; c.nrhs = nrhs; c.maxit = maxit;
    c.tol2 = tol * tol;
    c.g = ctx->g;
    c.S.scale = b.cgs; c.S.done = b.cgs + b.npad; c.S.iters = b.cgs + 2 * b.npad; c.S.r2 = b.cgs + 3 * b.npad;
    c.S.gamma = b.cgs + 4 * b.npad; c.S.alpha = b.cgs + 5 * b.npad; c.S.beta = b.cgs + 6 * b.npad;
    c.S.csp = b.cgs + 7 * b.npad; c.S.csr = b.cgs + 8 * b.npad;
    c.xpart = b.xpart; c.rpart = b.rpart; c.active = b.flags; c.err = b.flags + 1;
    return c;
}

// CGNR on the panel rcB -> yB for columns 0..nrhs-1 (zero columns stay zero).
// iters_out[n] += coarse iterations of column n.
int batched_coarse_solve(mg_ctx* ctx, int nrhs, double tol, int maxit, std::vector<double>& iters_out) {
    BatchWork& b = ctx->bw;
    TRY(ensure_embedding(ctx, ctx->full));
    CK(coarse_apply_tc_prepare(ctx->full.nc, b.npad));
    BatchCg c = batch_cg(ctx, tol, maxit, nrhs);
    {   // tile width from the autotuner (timed on the panel buffers once per shape)
        TcApplyArgs t{c.Aemb, c.p, c.q, c.nc, c.npad, 0, 0, c.g, nullptr, c.err, nullptr, c.bt, 0};
        c.nw = coarse_apply_tc_tune(t, ctx->st, &c.stages);
        CKL();
    }
    long long tolbits = 0;
    std::memcpy(&tolbits, &c.tol2, sizeof(tolbits));
    long long key[6] = {(long long)(size_t)c.Aemb, b.npad, nrhs, maxit, tolbits,
                        (ctx->full.nc * 1024 + c.nw) * 4 + c.stages};
    if (!b.graph || std::memcmp(key, b.graph_key, sizeof(key)) != 0) {
        if (b.graph) { cudaGraphExecDestroy(b.graph); b.graph = nullptr; }
        cudaGraph_t gr;
        CK(cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal));
        for (int j = 0; j < kBatchCheck; ++j) bcg_iteration(c, b.cap);
        CK(cudaStreamEndCapture(b.cap, &gr));
        // captured launches run only when the graph is replayed (counted there)
        launch_counter().fetch_sub(kBatchCheck * kBcgKernelsPerIteration, std::memory_order_relaxed);
        cudaError_t e = cudaGraphInstantiate(&b.graph, gr, 0);
        cudaGraphDestroy(gr);
        CK(e);
        std::memcpy(b.graph_key, key, sizeof(key));
    }
    PROF_BEGIN(MG_K_COARSE_SOLVE);
    bcg_start(c, ctx->st);
    CKL();
    int done_its = 0;
    for (;;) {
        CK(cudaGraphLaunch(b.graph, ctx->st));
        launch_counter().fetch_add(kBatchCheck * kBcgKernelsPerIteration, std::memory_order_relaxed);
        done_its += kBatchCheck;
        CK(cudaMemcpyAsync(b.h_flags, b.flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        if (b.h_flags[1]) return fail(ctx, MG_ERR_TIMEOUT, "batched coarse stencil: a bounded wait gave up");
        if (b.h_flags[0] == 0 || done_its >= maxit) break;
    }
    bcg_finish(c, ctx->st);
    PROF_END(MG_K_COARSE_SOLVE);
    CKL();
    CK(cudaMemcpyAsync(b.h_iters, c.S.iters, sizeof(double) * b.npad, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int n = 0; n < nrhs; ++n) iters_out[n] += b.h_iters[n];
    return MG_OK;
}

// b64 (internal layout) -> x64 for nrhs sources, FP32 inner precision
int solve_batched_impl(mg_ctx* ctx, int nrhs, mg_solve_info* infos) {
    TRY(ensure_work<float>(ctx));
    BatchWork& b = ctx->bw;
    const mg_params& p = ctx->prm;
    const CoarseLevel& L = ctx->full;
    const size_t n = nfine(ctx);
    const int K = b.K;
    const v2<float>* U = links<float>(ctx);
    std::vector<double> bnorm(nrhs), rnorm(nrhs), rcycle(nrhs), rel(nrhs, 1.0), coarse(nrhs, 0.0);
    std::vector<int> iters(nrhs, 0), restarts(nrhs, 0), status(nrhs, MG_ERR_NOT_CONVERGED), kk(nrhs, 0),
        active(nrhs, 1), cycle_end(nrhs, 0), mv(nrhs, 0);
    std::vector<double> mvb(nrhs, 0.0);   // bytes per site of the fine operator applications
    std::string why;                      // the first numeric failure, for the error message
    auto RR = [&](int r) {
        Reduce R = ctx->R;
        R.scal = b.scal + (size_t)r * S_COUNT;
        return R;
    };
    CK(cudaEventRecord(ctx->ev0, ctx->st));
    for (int r = 0; r < nrhs; ++r) {
        norm2<double>(b.b64 + r * n, n, S_NORM_A, RR(r), ctx->st);
        zero<double>(b.x64 + r * n, n, ctx->st);
        convert<double, float>(b.r32 + r * n, b.b64 + r * n, n, ctx->st);
    }
    CKL();
    CK(cudaMemcpyAsync(b.h_scal, b.scal, sizeof(double) * S_COUNT * nrhs, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int r = 0; r < nrhs; ++r) {
        bnorm[r] = std::sqrt(b.h_scal[(size_t)r * S_COUNT + S_NORM_A]);
        if (!std::isfinite(bnorm[r])) return fail(ctx, MG_ERR_NUMERIC, "right-hand side is not finite");
        rnorm[r] = rcycle[r] = bnorm[r];
        if (bnorm[r] == 0) { status[r] = MG_OK; active[r] = 0; rel[r] = 0; }
    }
    auto any_active = [&]() { for (int r = 0; r < nrhs; ++r) if (active[r]) return true; return false; };
    while (any_active()) {
        bool stepping = false;
        for (int r = 0; r < nrhs; ++r)
            if (active[r] && !cycle_end[r] && kk[r] < K && iters[r] < p.max_outer) stepping = true;
        if (stepping) {
            // restriction of every stepping source into its panel column
            CK(cudaMemsetAsync(b.rcB, 0, sizeof(float2) * (size_t)ctx->g.Vc * L.nc * b.npad, ctx->st));
            PROF_BEGIN(MG_K_RESTRICT);
            for (int r = 0; r < nrhs; ++r)
                if (active[r] && !cycle_end[r] && kk[r] < K && iters[r] < p.max_outer)
                    restrict_<float>(b.rcB, L.P32, b.r32 + r * n, L.nv, ctx->g, ctx->st, b.npad, r);
            PROF_END(MG_K_RESTRICT);
            CKL();
            TRY(batched_coarse_solve(ctx, nrhs, p.coarse_tol, p.max_coarse, coarse));
            for (int r = 0; r < nrhs; ++r) {
                if (!(active[r] && !cycle_end[r] && kk[r] < K && iters[r] < p.max_outer)) continue;
                Reduce Rr = RR(r);
                v2<float>* zk = b.Z + ((size_t)r * K + kk[r]) * n;
                v2<float>* Pr = b.Pk + (size_t)r * K * n;
                PROF_BEGIN(MG_K_PROLONG);
                prolong<float>(zk, L.P32, b.yB, L.nv, ctx->g, ctx->st, b.npad, r);
                PROF_END(MG_K_PROLONG);
                {
                    Counters scnt;
                    TRY(smooth<float>(ctx, b.r32 + r * n, zk, Rr, scnt));
                    mv[r] += scnt.matvecs;
                    mvb[r] += scnt.site_bytes;
                }
                PROF_BEGIN(MG_K_DSLASH);
                dslash<float>(DS_PLAIN, Pr + (size_t)kk[r] * n, zk, U, zk, ctx->g, ctx->mass, 0.0, 0, Rr, ctx->st);
                PROF_END(MG_K_DSLASH);
                mv[r] += 1;
                mvb[r] += kDslashBytesF32;
                PROF_BEGIN(MG_K_KRYLOV);
                if (kk[r] > 0) {
                    gcr_multidot<float>(Pr, n, kk[r], Rr, ctx->st);
                    gcr_orth_norm<float>(Pr, n, kk[r], Rr, ctx->st);
                } else {
                    norm2<float>(Pr, n, S_GCR_PN2, Rr, ctx->st);
                }
                gcr_cdot<float>(Pr, b.r32 + r * n, n, kk[r], Rr, ctx->st);
                gcr_update<float>(Pr, b.r32 + r * n, n, kk[r], Rr, ctx->st);
                PROF_END(MG_K_KRYLOV);
                CKL();
            }
            CK(cudaMemcpyAsync(b.h_scal, b.scal, sizeof(double) * S_COUNT * nrhs, cudaMemcpyDeviceToHost, ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
            for (int r = 0; r < nrhs; ++r) {
                if (!(active[r] && !cycle_end[r] && kk[r] < K && iters[r] < p.max_outer)) continue;
                const double* sc = b.h_scal + (size_t)r * S_COUNT;
                ++kk[r];
                ++iters[r];
                double pn = sc[S_GCR_PN2];
                if (!(pn > 0) || !std::isfinite(pn)) {
                    status[r] = MG_ERR_NUMERIC;
                    active[r] = 0;
                    if (why.empty())
                        why = "source " + std::to_string(r) + ": GCR breakdown, |D z|^2 = " + std::to_string(pn) +
                              " at outer iteration " + std::to_string(iters[r]);
                    continue;
                }
                rnorm[r] = std::sqrt(sc[S_GCR_R2]);
                if (rnorm[r] <= p.tol * bnorm[r] || (p.delta > 0 && rnorm[r] <= p.delta * rcycle[r]) || kk[r] >= K ||
                    iters[r] >= p.max_outer)
                    cycle_end[r] = 1;
            }
        }
        // restart every source that closed its cycle once no source is still stepping in it
        bool all_closed = true;
        for (int r = 0; r < nrhs; ++r)
            if (active[r] && !cycle_end[r] && kk[r] < K && iters[r] < p.max_outer) all_closed = false;
        if (!all_closed) continue;
        for (int r = 0; r < nrhs; ++r) {
            if (!active[r]) continue;
            const double* sc = b.h_scal + (size_t)r * S_COUNT;
            int k = kk[r];
            auto Rr = [&](int j, int c) { return sc + S_GCR_R + 2 * (c * K_MAX + j); };
            GcrCoef y{};
            for (int i = k - 1; i >= 0; --i) {
                double sr = sc[S_GCR_C + 2 * i], si = sc[S_GCR_C + 2 * i + 1];
                for (int j = i + 1; j < k; ++j) {
                    const double* q = Rr(i, j);
                    sr -= q[0] * y.c[2 * j] - q[1] * y.c[2 * j + 1];
                    si -= q[0] * y.c[2 * j + 1] + q[1] * y.c[2 * j];
                }
                const double* dd = Rr(i, i);
                double den = dd[0] * dd[0] + dd[1] * dd[1];
                y.c[2 * i] = (sr * dd[0] + si * dd[1]) / den;
                y.c[2 * i + 1] = (si * dd[0] - sr * dd[1]) / den;
            }
            Reduce R = RR(r);
            PROF_BEGIN(MG_K_KRYLOV);
            gcr_xupdate<float>(b.x64 + r * n, b.Z + (size_t)r * K * n, n, k, y, ctx->st);
            PROF_END(MG_K_KRYLOV);
            PROF_BEGIN(MG_K_TRUE_RESIDUAL);
            dslash<double>(DS_XMY_NORM, ctx->r64, b.x64 + r * n, ctx->U64, b.b64 + r * n, ctx->g, ctx->mass, 0.0, S_NORM_B,
                           R, ctx->st);
            PROF_END(MG_K_TRUE_RESIDUAL);
            convert<double, float>(b.r32 + r * n, ctx->r64, n, ctx->st);
            mv[r] += 1;
            mvb[r] += kDslashBytesF64;
            CKL();
        }
        CK(cudaMemcpyAsync(b.h_scal, b.scal, sizeof(double) * S_COUNT * nrhs, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        for (int r = 0; r < nrhs; ++r) {
            if (!active[r]) continue;
            ++restarts[r];
            rnorm[r] = std::sqrt(b.h_scal[(size_t)r * S_COUNT + S_NORM_B]);
            rel[r] = rnorm[r] / bnorm[r];
            kk[r] = 0;
            cycle_end[r] = 0;
            rcycle[r] = rnorm[r];
            if (!std::isfinite(rel[r])) {
                status[r] = MG_ERR_NUMERIC;
                active[r] = 0;
                if (why.empty())
                    why = "source " + std::to_string(r) + ": non-finite true residual after outer iteration " +
                          std::to_string(iters[r]);
            }
            else if (rel[r] <= p.tol) { status[r] = MG_OK; active[r] = 0; }
            else if (iters[r] >= p.max_outer) { status[r] = MG_ERR_NOT_CONVERGED; active[r] = 0; }
        }
    }
    CK(cudaEventRecord(ctx->ev1, ctx->st));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    int worst = MG_OK;
    for (int r = 0; r < nrhs; ++r) {
        if (infos) {
            infos[r].outer_iters = iters[r];
            infos[r].coarse_iters = (int)coarse[r];
            infos[r].fine_matvecs = mv[r];
            infos[r].restarts = restarts[r];
            infos[r].true_rel_res = rel[r];
            infos[r].solve_ms = ms;
            infos[r].setup_ms = ctx->setup_ms;
            infos[r].dslash_bytes = mvb[r] * (double)ctx->g.V;
            infos[r].status = status[r];
        }
        if (status[r] == MG_ERR_NUMERIC) worst = MG_ERR_NUMERIC;
        else if (status[r] == MG_ERR_NOT_CONVERGED && worst == MG_OK) worst = MG_ERR_NOT_CONVERGED;
    }
    if (worst == MG_ERR_NUMERIC) ctx->err = "batched solve: " + why;
    if (worst == MG_ERR_NOT_CONVERGED) ctx->err = "max_outer reached for a batched source";
    return worst;
}

}  // namespace

extern "C" {

int mg_solve_batched_device(mg_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, mg_solve_info* infos) {
    TRY(need_cycle(ctx));
    if (!b_dev || !x_dev || nrhs <= 0) return fail(ctx, MG_ERR_INVALID_ARG, "null buffer or nrhs <= 0");
    size_t n = nfine(ctx);
    if (ctx->prm.prec_inner == MG_FP64) {   // FP64 inner precision: the sources one after another
        int worst = MG_OK;
        for (int r = 0; r < nrhs; ++r) {
            int st = mg_solve_device(ctx, b_dev + 2 * r * n, x_dev + 2 * r * n, infos ? infos + r : nullptr);
            if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return st;
            if (st != MG_OK) worst = st;
        }
        return worst;
    }
    if (nrhs > 256) return fail(ctx, MG_ERR_INVALID_ARG, "at most 256 sources per batch");
    if (ctx->prm.levels != 2) return fail(ctx, MG_ERR_INVALID_ARG, "the batched solve runs the two-level cycle");
    if (!coarse_apply_tc_supported(ctx->full.nc, round16(nrhs)))
        return fail(ctx, MG_ERR_INVALID_ARG, "batched coarse stencil needs 2*nvec a multiple of 16 and <= 128");
    TRY(ensure_batch(ctx, nrhs));
    for (int r = 0; r < nrhs; ++r)
        spinor_to_internal<double>(ctx->bw.b64 + r * n, (const double2*)b_dev + r * n, ctx->g, ctx->st);
    CKL();
    int st = solve_batched_impl(ctx, nrhs, infos);
    if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return st;
    for (int r = 0; r < nrhs; ++r)
        spinor_from_internal<double>((double2*)x_dev + r * n, ctx->bw.x64 + r * n, ctx->g, ctx->st);
    CKL();
    CK(cudaStreamSynchronize(ctx->st));
    return st;
}

int mg_solve_batched(mg_ctx* ctx, const double* b, double* x, int nrhs, mg_solve_info* infos) {
    TRY(need_cycle(ctx));
    if (!b || !x || nrhs <= 0) return fail(ctx, MG_ERR_INVALID_ARG, "null buffer or nrhs <= 0");
    size_t n = nfine(ctx);
    double2 *db = nullptr, *dx = nullptr;
    TRY(dalloc(ctx, &db, sizeof(double2) * n * nrhs));
    TRY(dalloc(ctx, &dx, sizeof(double2) * n * nrhs));
    CK(cudaMemcpyAsync(db, b, sizeof(double2) * n * nrhs, cudaMemcpyHostToDevice, ctx->st));
    int st = mg_solve_batched_device(ctx, (const double*)db, (double*)dx, nrhs, infos);
    if (st == MG_OK || st == MG_ERR_NOT_CONVERGED) {
        CK(cudaMemcpyAsync(x, dx, sizeof(double2) * n * nrhs, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    // release the staging buffers of this call
    for (void* q : {(void*)db, (void*)dx}) {
        for (size_t i = 0; i < ctx->allocs.size(); ++i)
            if (ctx->allocs[i] == q) { ctx->allocs.erase(ctx->allocs.begin() + i); break; }
        cudaFree(q);
    }
    return st;
}

int mg_time_coarse_batched(mg_ctx* ctx, int nrhs, int reps, double* ms_per_launch, double* bytes_per_launch,
                           double* flops_per_launch) {
    TRY(need_level(ctx));
    if (nrhs <= 0 || nrhs > 256 || reps <= 0 || !ms_per_launch) return MG_ERR_INVALID_ARG;
    CoarseLevel& L = ctx->full;
    const int npad = round16(nrhs);
    if (!coarse_apply_tc_supported(L.nc, npad)) return fail(ctx, MG_ERR_INVALID_ARG, "unsupported shape");
    const size_t npanel = (size_t)ctx->g.Vc * L.nc * npad;
    float2 *pa = nullptr, *pb = nullptr;
    int* err = nullptr;
    __half* bt = nullptr;
    TRY(dalloc(ctx, &pa, sizeof(float2) * npanel));
    TRY(dalloc(ctx, &pb, sizeof(float2) * npanel));
    TRY(dalloc(ctx, &err, sizeof(int) * 4));
    TRY(dalloc(ctx, &bt, tc_split_bytes(L.nc, npad, ctx->g.Vc)));
    auto release = [&]() {
        for (void* q : {(void*)pa, (void*)pb, (void*)err, (void*)bt}) {
            for (size_t i = 0; i < ctx->allocs.size(); ++i)
                if (ctx->allocs[i] == q) { ctx->allocs.erase(ctx->allocs.begin() + i); break; }
            cudaFree(q);
        }
    };
    int st = MG_OK;
    do {
        if ((st = ensure_embedding(ctx, L)) != MG_OK) break;
        if (cudaMemsetAsync(err, 0, sizeof(int) * 4, ctx->st) != cudaSuccess ||
            cudaMemsetAsync(pb, 0, sizeof(float2) * npanel, ctx->st) != cudaSuccess ||
            coarse_apply_tc_prepare(L.nc, npad) != cudaSuccess) { st = fail(ctx, MG_ERR_CUDA, "probe setup"); break; }
        // a zero panel (the values do not change the work or its timing)
        panel_pack(pa, nullptr, (long long)ctx->g.Vc * L.nc, 0, npad, ctx->st);
        TcApplyArgs a{L.Aemb, pa, pb, L.nc, npad, 0, 0, ctx->g, nullptr, err, nullptr, bt, 0};
        a.nw = coarse_apply_tc_tune(a, ctx->st, &a.stages);
        for (int i = 0; i < 2; ++i) coarse_apply_tc(a, ctx->st);
        cudaEventRecord(ctx->ev0, ctx->st);
        for (int i = 0; i < reps; ++i) coarse_apply_tc(a, ctx->st);
        cudaEventRecord(ctx->ev1, ctx->st);
        if (cudaEventSynchronize(ctx->ev1) != cudaSuccess) { st = fail(ctx, MG_ERR_CUDA, "probe launch"); break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        int h_err = 0;
        cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
        if (h_err) { st = fail(ctx, MG_ERR_TIMEOUT, "batched coarse stencil: a bounded wait gave up"); break; }
        *ms_per_launch = (double)ms / reps;
        const double K = 2.0 * L.nc;
        // algorithmic: the FP16 embedded operator once, the FP32 panel read once and written once
        if (bytes_per_launch) *bytes_per_launch = (double)ctx->g.Vc * 9 * K * K * 2 + 2.0 * npanel * sizeof(float2);
        // useful work: 9 complex nc x nc blocks times nrhs columns per aggregate (8 real flops per complex MAC)
        if (flops_per_launch) *flops_per_launch = 8.0 * 9 * L.nc * (double)L.nc * ctx->g.Vc * nrhs;
    } while (false);
    release();
    return st;
}

int mg_apply_coarse_batched(mg_ctx* ctx, const double* x, double* y, int nrhs, int dagger, int impl) {
    TRY(need_level(ctx));
    if (!x || !y || nrhs <= 0 || nrhs > 256) return fail(ctx, MG_ERR_INVALID_ARG, "bad buffers or nrhs");
    const CoarseLevel& L = ctx->full;
    int npad = round16(nrhs);
    long long rows = (long long)ctx->g.Vc * L.nc;
    size_t nin = (size_t)rows * nrhs, npanel = (size_t)rows * npad;
    double2 *hin = nullptr, *hout = nullptr, *p64a = nullptr, *p64b = nullptr;
    float2 *pa = nullptr, *pb = nullptr;
    // each source scaled to max |x| = 1 (the FP16 panel of the tensor-core path has
    // no subnormal headroom), scaled back afterwards
    std::vector<double> scale(nrhs, 1.0), xs((size_t)2 * nin);
    for (int r = 0; r < nrhs; ++r) {
        double mx = 0;
        for (long long i = 0; i < 2 * rows; ++i) mx = std::max(mx, std::fabs(x[(size_t)r * 2 * rows + i]));
        scale[r] = mx > 0 ? mx : 1.0;
        for (long long i = 0; i < 2 * rows; ++i) xs[(size_t)r * 2 * rows + i] = x[(size_t)r * 2 * rows + i] / scale[r];
    }
    TRY(dalloc(ctx, &hin, sizeof(double2) * nin));
    TRY(dalloc(ctx, &hout, sizeof(double2) * nin));
    CK(cudaMemcpyAsync(hin, xs.data(), sizeof(double2) * nin, cudaMemcpyHostToDevice, ctx->st));
    std::vector<void*> tmp = {hin, hout};
    int st = MG_OK;
    if (impl == 0) {
        if (!coarse_apply_tc_supported(L.nc, npad)) return fail(ctx, MG_ERR_INVALID_ARG, "unsupported shape");
        TRY(dalloc(ctx, &pa, sizeof(float2) * npanel));
        TRY(dalloc(ctx, &pb, sizeof(float2) * npanel));
        tmp.push_back(pa);
        tmp.push_back(pb);
        TRY(dalloc(ctx, &p64a, sizeof(int) * 4));   // error flag
        tmp.push_back(p64a);
        __half* bt = nullptr;
        TRY(dalloc(ctx, &bt, tc_split_bytes(L.nc, npad, ctx->g.Vc)));
        tmp.push_back(bt);
        CK(cudaMemsetAsync(p64a, 0, sizeof(int) * 4, ctx->st));
        TRY(ensure_embedding(ctx, ctx->full));
        panel_pack(pa, hin, rows, nrhs, npad, ctx->st);
        CK(coarse_apply_tc_prepare(L.nc, npad));
        TcApplyArgs a{L.Aemb, pa, pb, L.nc, npad, 0, dagger ? 1 : 0, ctx->g, nullptr, (int*)p64a, nullptr, bt, 0};
        a.nw = coarse_apply_tc_tune(a, ctx->st, &a.stages);
        CK(coarse_apply_tc(a, ctx->st));
        panel_unpack(hout, pb, rows, nrhs, npad, ctx->st);
        int err = 0;
        CK(cudaMemcpyAsync(&err, p64a, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        if (err) st = fail(ctx, MG_ERR_TIMEOUT, "batched coarse stencil: a bounded wait gave up");
    } else {
        TRY(dalloc(ctx, &p64a, sizeof(double2) * npanel));
        TRY(dalloc(ctx, &p64b, sizeof(double2) * npanel));
        tmp.push_back(p64a);
        tmp.push_back(p64b);
        panel_pack64(p64a, hin, rows, nrhs, npad, ctx->st);
        coarse_apply_batched_simt<double>(p64b, L.A64, p64a, L.nc, npad, dagger != 0, ctx->g, ctx->st);
        panel_unpack64(hout, p64b, rows, nrhs, npad, ctx->st);
    }
    CKL();
    if (st == MG_OK) {
        CK(cudaMemcpyAsync(y, hout, sizeof(double2) * nin, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        for (int r = 0; r < nrhs; ++r)
            for (long long i = 0; i < 2 * rows; ++i) y[(size_t)r * 2 * rows + i] *= scale[r];
    }
    for (void* q : tmp) {
        for (size_t i = 0; i < ctx->allocs.size(); ++i)
            if (ctx->allocs[i] == q) { ctx->allocs.erase(ctx->allocs.begin() + i); break; }
        cudaFree(q);
    }
    return st;
}

}  // extern "C"

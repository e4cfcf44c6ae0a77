// Host-side launchers of the library's kernels (internal, not part of the C-ABI).
#pragma once
#include <mutex>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>

#include "mg_common.cuh"

namespace wmg {

// Count of kernel launches issued by this library (all contexts, all threads).
std::atomic<long long>& launch_counter();
// SM count of the current device (looked up once per device)
int device_sm_count();
inline void note_launch() { launch_counter().fetch_add(1, std::memory_order_relaxed); }

// Scratch used by the single-pass grid reductions: per-block partial sums and
// an arrival counter that the last block resets to zero.
struct Reduce {
    double* partials;      // partial_bytes bytes (at least kReducePartialsBytes)
    unsigned int* ticket;  // one zeroed counter
    double* scal;          // device scalars, S_COUNT doubles (ScalarSlot)
    size_t partial_bytes;  // capacity of partials
};
// partial-sum buffer for a lattice of V sites: the widest per-block reduction of
// the per-site kernels (32 floats per 128 sites) or kReducePartialsBytes
inline size_t reduce_partial_bytes(long long V) {
    const size_t per_site = (size_t)((V + 127) / 128) * 32 * sizeof(float);
    return per_site > kReducePartialsBytes ? per_site : kReducePartialsBytes;
}

// ---------------------------------------------------------------- layout conversion
template <typename T> void spinor_to_internal(v2<T>* out, const double2* in_lex, const Geom& g, cudaStream_t st);
template <typename T> void spinor_from_internal(double2* out_lex, const v2<T>* in, const Geom& g, cudaStream_t st);
template <typename T> void links_to_internal(v2<T>* out, const double2* in_lex, const Geom& g, cudaStream_t st);
template <typename Tin, typename Tout> void convert(v2<Tout>* out, const v2<Tin>* in, size_t n, cudaStream_t st);

// ---------------------------------------------------------------- fine operator (eq. 2)
enum DslashMode { DS_PLAIN = 0, DS_XMY = 1, DS_XMY_NORM = 2, DS_MRDOT = 3 };
// DS_PLAIN:     out = D in
// DS_XMY:       out = src - D in
// DS_XMY_NORM:  out = src - D in, scal[slot] = ||out||^2
// DS_MRDOT:     out = D in, scal[S_MR_ALPHA] = omega <out,in> / <out,out>
template <typename T>
void dslash(int mode, v2<T>* out, const v2<T>* in, const v2<T>* U, const v2<T>* src, const Geom& g, double mass,
            double omega, int slot, const Reduce& R, cudaStream_t st);

// ---------------------------------------------------------------- fine / generic BLAS (n complex)
template <typename T> void zero(v2<T>* x, size_t n, cudaStream_t st);
template <typename T> void norm2(const v2<T>* x, size_t n, int slot, const Reduce& R, cudaStream_t st);
template <typename T> void dot(const v2<T>* x, const v2<T>* y, size_t n, int slot, const Reduce& R, cudaStream_t st);
template <typename T> void scale(v2<T>* x, size_t n, double s, cudaStream_t st);
// y += a x with a a host constant
template <typename T> void axpy(v2<T>* y, const v2<T>* x, size_t n, double ar, double ai, cudaStream_t st);
// MR update: e += alpha r; r -= alpha q (if update_r), alpha = scal[S_MR_ALPHA]
template <typename T>
void mr_update(v2<T>* e, v2<T>* r, const v2<T>* q, size_t n, bool update_r, const Reduce& R, cudaStream_t st);
// normalise x in place by 1/sqrt(scal[slot])
template <typename T> void normalize_dev(v2<T>* x, size_t n, int slot, const Reduce& R, cudaStream_t st);

// ---------------------------------------------------------------- GCR (K_MAX basis vectors)
// R[j][k] = <p_j, p_k> for j < k  (p_j = basis + j*n)
template <typename T> void gcr_multidot(const v2<T>* basis, size_t n, int k, const Reduce& R, cudaStream_t st);
// p_k -= sum_{j<k} R[j][k] p_j ; scal[S_GCR_PN2] = ||p_k||^2
template <typename T> void gcr_orth_norm(v2<T>* basis, size_t n, int k, const Reduce& R, cudaStream_t st);
// R[k][k] = ||p_k||; c_k = <p_k, r>/||p_k||
template <typename T> void gcr_cdot(const v2<T>* basis, const v2<T>* r, size_t n, int k, const Reduce& R, cudaStream_t st);
// p_k /= ||p_k||; r -= c_k p_k; scal[S_GCR_R2] = ||r||^2
template <typename T> void gcr_update(v2<T>* basis, v2<T>* r, size_t n, int k, const Reduce& R, cudaStream_t st);
// x (FP64) += sum_j y_j Z_j
struct GcrCoef { double c[2 * K_MAX]; };
template <typename T>
void gcr_xupdate(double2* x, const v2<T>* Z, size_t n, int k, const GcrCoef& y, cudaStream_t st);
// GMRES(k) smoother pieces: normalise basis[k] by sqrt(scal[S_GCR_PN2]) and record
// it as h_{k,k-1}; solve the small least-squares problem (omega y -> S_GCR_C);
// z += sum_j c_j basis[j]
template <typename T> void gmres_normalize(v2<T>* basis, size_t n, int k, const Reduce& R, cudaStream_t st);
void gmres_ls(const Reduce& R, int k, double omega, cudaStream_t st);
template <typename T> void multi_axpy(v2<T>* z, const v2<T>* basis, size_t n, int k, const Reduce& R, cudaStream_t st);

// ---------------------------------------------------------------- transfer / coarse
// P64[X][s][i][6][l] from prototypes V[i][X][12][l]; *status = 1 on rank deficiency
void block_orthonormalize(double2* P, const double2* V, int nv, const Geom& g, int* d_status, cudaStream_t st);
// coarse vector entry (X, a) lives at index (X*2nv + a)*cstride + coff (1, 0: plain coarse vector;
// npad, n: column n of an RHS panel)
template <typename T>
void restrict_(v2<T>* rc, const v2<T>* P, const v2<T>* r, int nv, const Geom& g, cudaStream_t st, int cstride = 1,
               int coff = 0);
template <typename T>
void prolong(v2<T>* e, const v2<T>* P, const v2<T>* yc, int nv, const Geom& g, cudaStream_t st, int cstride = 1,
             int coff = 0);
// A64 (column-major blocks) = P^dag D P; Aself scratch of Vc*8*nc*nc complex
void coarse_build(double2* A, double2* Aself, const double2* P, const double2* U, int nv, double mass, const Geom& g,
                  cudaStream_t st);
// same with FP32 products (P, U in FP32), per-chunk sums added in FP64
void coarse_build_f32(double2* A, double2* Aself, const float2* P, const float2* U, int nv, double mass, const Geom& g,
                      cudaStream_t st);
void coarse_shift_mass(double2* A, int nc, double dm, const Geom& g, cudaStream_t st);
// y = D_c x (dag: sigma3 D_c sigma3 x); with slot >= 0 also scal[slot] = ||y||^2
template <typename T>
void coarse_apply(v2<T>* y, const v2<T>* A, const v2<T>* x, int nc, bool dag, int slot, const Geom& g, const Reduce& R,
                  cudaStream_t st);
// block-orthonormal prolongator to the boundary null-vector layout
void prolongator_to_boundary(double2* out, const double2* P, int nv, const Geom& g, cudaStream_t st);
// boundary <-> internal coarse operator ([X][d][a][b] row-major <-> [X][d][b][a])
void coarse_op_transpose(double2* out, const double2* in, int nc, int Vc, cudaStream_t st);

// CGNR (CGLS) on D_c with device-side control: the kernels become no-ops once
// scal[S_CG_DONE] is set.
template <typename T>
void cg_init(v2<T>* y, v2<T>* r, const v2<T>* rc, size_t n, double tol, int maxit, const Reduce& R, cudaStream_t st);
template <typename T>
void cg_first_direction(v2<T>* s, v2<T>* p, const v2<T>* r, const v2<T>* A, int nc, const Geom& g, const Reduce& R,
                        cudaStream_t st);
template <typename T>
void cg_step(v2<T>* y, v2<T>* r, v2<T>* s, v2<T>* p, v2<T>* q, const v2<T>* A, int nc, const Geom& g, const Reduce& R,
             cudaStream_t st);

// Whole CGNR solve in one cooperative launch (bounded-wait grid barriers, two per iteration).
// Writes scal[S_CG_ITERS, S_CG_R2, S_CG_RC2], adds the count to scal[S_CG_TOTAL];
// *err = 1 if a barrier wait gave up.
template <typename T> struct CgnrArgs {
    v2<T>* y;
    v2<T>* r;              // r and r1, p and p1: double buffers
    v2<T>* r1;
    v2<T>* s;
    v2<T>* p;
    v2<T>* p1;
    v2<T>* q;
    const v2<T>* A;
    const __half2* A16;    // optional FP16 operator (T = float): A = s16[X*9+d] * A16
    const float* s16;
    const int* nbr;        // coarse neighbour table [Vc][9]
    const v2<T>* rc;
    int nc;
    int xpb;               // aggregates per CTA (set by the launcher)
    Geom g;
    double tol2;
    int maxit;
    double* partials;      // >= 4 * (co-resident CTAs) doubles
    unsigned int* bar;     // 2 zeroed counters
    double* scal;
    int* err;
};
template <typename T> cudaError_t cgnr_persistent(const CgnrArgs<T>& args, cudaStream_t st);
void coarse_neighbour_table(int* nbr, const Geom& g, cudaStream_t st);

// FP16 storage of fine spinors (kernels_half.cu): v[X][6][l] holds components
// (2j, 2j+1) as two __half2 (value / s[X][l]); FP16 links U16[mu][X][5][l]
struct HalfSpinor {
    uint2* v;
    float* s;
};
struct ConstHalfSpinor {
    const uint2* v;
    const float* s;
    ConstHalfSpinor(const uint2* v_, const float* s_) : v(v_), s(s_) {}
    ConstHalfSpinor(HalfSpinor h) : v(h.v), s(h.s) {}
};
void links_to_half(uint2* U16, const float2* U32, const Geom& g, cudaStream_t st);
// the FP32 links in the dslash's paired layout (36 float2 per site): the dslash<float>
// launchers take this array, the coarse build and the FP16 copy the plain one
void links_pair(float2* out, const float2* U32, const Geom& g, cudaStream_t st);
void to_half(HalfSpinor h, const float2* x, const Geom& g, cudaStream_t st);
void from_half(float2* x, ConstHalfSpinor h, const Geom& g, cudaStream_t st);
// in_norm (device scalar, or nullptr): the input's site scales times the
// float *in_norm (an Arnoldi vector normalised through its stored 1 / |v|)
void dslash_h_plain(HalfSpinor out, ConstHalfSpinor in, const uint2* U16, const Geom& g, double mass, cudaStream_t st,
                    const double* in_norm = nullptr);
// out = src - D in (in FP32)
void dslash_h_xmy(HalfSpinor out, const float2* in, const uint2* U16, const float2* src, const Geom& g, double mass,
                  cudaStream_t st);
// out = D in, scal[S_MR_ALPHA..+1] = omega <out, in> / |out|^2 of the stored out
void dslash_h_mrdot(HalfSpinor out, ConstHalfSpinor in, const uint2* U16, const Geom& g, double mass, double omega,
                    const Reduce& R, cudaStream_t st);
// GMRES basis in FP16 storage: B[j] / S[j] = vector j in the HalfSpinor layout
// (6 V pair words, V site scales each); dots of basis[k] with basis[j < k] into the
// Hessenberg scalars, Gram-Schmidt update of basis[k] (and its norm^2 into
// S_GCR_PN2), normalisation by rescaling the site scales, z += sum c_j basis[j]
void h_multidot(const uint2* B, const float* S, const Geom& g, int k, const Reduce& R, cudaStream_t st);
void h_orth(uint2* B, float* S, const Geom& g, int k, const Reduce& R, cudaStream_t st);
void h_multi_axpy(float2* z, const uint2* B, const float* S, const Geom& g, int k, const Reduce& R, cudaStream_t st);
// e += alpha r; r -= alpha q when update_r (alpha from scal[S_MR_ALPHA])
void mr_update_h(float2* e, HalfSpinor r, ConstHalfSpinor q, const Geom& g, bool update_r, const Reduce& R,
                 cudaStream_t st);

// Coarse CGLS with the operator on chip (kernels_cgls.cu).  The operator rows
// of each aggregate are cut into units of `ru` rows, Au[X*H + h][d][b][a].
struct CglsShape {
    int ru;          // operator rows per unit (divides nc)
    int grid;        // CTAs, at most one per SM
    int nu_max;      // units of the busiest CTA
    int nx_max;      // aggregates the units of one CTA can touch
    int slots;       // unit slots in shared memory
    int wave;        // units per wave
    int groups;      // slot groups in flight (streamed mode)
    int resident;    // 1: every CTA keeps all its units in shared memory
    int stride;      // bytes between slots
    int slot_off;    // byte offset of slot 0 in dynamic shared memory
    int red_n;       // complex entries per reduction buffer
    int tm;          // the operator in tensor memory (all 512 columns of the SM): 1 products on the
                     // CUDA cores, 2 products on the tensor cores (tcgen05.mma, A from TMEM)
    int tm_chunks;   // 32-column TMEM chunks per thread (tm 1)
    int own_off;     // byte offset of the own-row vectors of the tagged form in shared memory (0: global)
    int bt_off;      // tm 2: byte offset of the FP16 hi/lo operand tile (MMA B) in shared memory
    int mma_lbo;     // tm 2: its byte distance between core matrices adjacent in K
    int rop_off;     // tm 2: byte offset of the rows beyond the 128 MMA rows (FP16 operator, shared memory)
    int rem_max;     // tm 2: those rows of the busiest CTA
    int mma_acc;     // tm 2: accumulators (32 TMEM columns each) the K steps alternate over
    size_t smem;     // dynamic shared memory per CTA
};
enum { CGLS_AUTO = 0, CGLS_STREAM = 2, CGLS_SMEM = 3, CGLS_TMEM_CORES = 4 };
// iteration form of the on-chip CGLS: two grid-wide exchanges per iteration, or
// the Chronopoulos-Gear form with one exchange and epoch-tagged shared vectors
enum { CGLS_TEXTBOOK = 0, CGLS_CG_TAGGED = 1 };
// latency probes on the same launch shape (maxit rounds, no arithmetic
// dependence on the results): the two tagged stencils of one Chronopoulos-Gear
// iteration without its exchange, or its exchange alone
enum { CGLS_PROBE_STENCILS = 2, CGLS_PROBE_EXCHANGE = 3 };
struct CglsArgs {
    const void* Au;        // float2 or __half2 units
    const float* su;       // FP16 block scales [X][d]; nullptr selects the FP32 operator
    const int* nbr;        // coarse neighbour table [Vc][9]
    const float2* rc;
    float2 *y, *r, *r1, *s, *p, *p1, *q;
    int nc;
    Geom g;
    float tol2;
    int maxit;
    unsigned long long* xch;   // exchange slots, kXchWords words
    unsigned int epoch0;       // first epoch of this launch; 2 * maxit + 4 are reserved
    int form;                  // CGLS_TEXTBOOK or CGLS_CG_TAGGED
    unsigned long long* tag;   // CGLS_CG_TAGGED: epoch-tagged s and u, 4 * Vc * nc words
    double* scal;
    int* err;                  // error flag (zeroed before the launch)
    CglsShape sh;
};
constexpr int kXchMaxGrid = 256;
// exchange slots [parity 2][value 3][grid][16]
constexpr size_t kXchWords = (size_t)2 * 3 * kXchMaxGrid * 16;
bool cgls_shape(int nc, int Vc, bool h16, int mode, CglsShape* out);
// Not for graph capture: every launch takes a fresh epoch range from the host.
void coarse_pack_units(void* Au, float* su, const double2* A, int nc, int ru, int Vc, bool h16, cudaStream_t st);
cudaError_t cgls_onchip(const CglsArgs& args, cudaStream_t st);
// ---------------------------------------------------------------- red-black preconditioned CG
// checkerboard geometry: Vh = V / 2 sites per parity, cb index = lex >> 1
struct EoGeom {
    int L[4];
    int Lh0;        // L[0] / 2
    long long Vh;
    int tap;
};
// epilogue flags of the half-lattice hop
enum EoFlags { EO_PLAIN = 0, EO_SRC = 1, EO_SELF = 2, EO_ACC = 4, EO_NORM = 8, EO_G5IN = 16, EO_G5H = 32, EO_SKIP = 64 };
// device scalar slots of the CG
struct EoCgSlots {
    int gamma, q2, r2, tol2, done, iters;
};
template <typename T>
void eo_hop(int flags, v2<T>* out, const v2<T>* in, const v2<T>* src, const v2<T>* self, const void* U,
            const EoGeom& e, int p, double c_src, double c_self, double c_h, int slot, int done_slot, const Reduce& R,
            cudaStream_t st);
template <typename T>
void eo_cg_update1(v2<T>* x, v2<T>* r, const v2<T>* p, const v2<T>* q, long long n, const EoCgSlots& s, int iter,
                   const Reduce& R, cudaStream_t st);
template <typename T>
void eo_cg_update2(v2<T>* p, const v2<T>* sv, long long n, int gamma_old, int gamma_new, int done, const Reduce& R,
                   cudaStream_t st);
template <typename T> void eo_spinor_pack(v2<T>* out, const double2* in, const EoGeom& e, cudaStream_t st);
template <typename T> void eo_spinor_unpack(double2* out, const v2<T>* in, const EoGeom& e, cudaStream_t st);
void eo_links_pack(double2* U64, float2* U32, const double2* Uint, const Geom& g, const EoGeom& e, cudaStream_t st);

// ---------------------------------------------------------------- level 2 (three-level method)
// g2: the level-1 lattice (L) cut into level-2 aggregates (B), Lc = level-2 lattice
void block_orthonormalize_l2(double2* P2, const double2* V2, int nv1, int nv2, const Geom& g2, int* status,
                             cudaStream_t st);
template <typename T>
void restrict_l2(v2<T>* r2, const v2<T>* P2, const v2<T>* r1, int nv1, int nv2, const Geom& g2, cudaStream_t st);
template <typename T>
void prolong_l2(v2<T>* e1, const v2<T>* P2, const v2<T>* y2, int nv1, int nv2, const Geom& g2, cudaStream_t st);
bool build_l2_supported(int nv1, int nv2);
cudaError_t coarse_build_l2(double2* A2, const double2* P2, const double2* A1, int nv1, int nv2, const Geom& g1,
                            const Geom& g2, cudaStream_t st);

// ---------------------------------------------------------------- learned setup (parallel-transport network)
cudaError_t nn_layer(float2* out, const float2* in, const float2* W, const float2* U, const Geom& g, int cin, int cout,
                     cudaStream_t st);
int nn_wgrad_blocks(const Geom& g);
cudaError_t nn_wgrad(double2* G, float2* part, const float2* gout, const float2* in, const float2* U, const Geom& g,
                     int cin, int cout, double scale, cudaStream_t st);
void nn_seed(float2* gout, const float2* r, const float2* v, size_t n, const double* scal, int vslot, int rslot,
             cudaStream_t st);
void nn_adam(float2* W, double2* Wm, const double2* G, double2* m, double2* v, int n, double lr, double b1, double b2,
             double eps, int t, cudaStream_t st);
void nn_adjoint_weights(float2* Wt, const float2* W, int cin, int cout, cudaStream_t st);

// Orders this process's TMEM-kernel launches across streams: construct before
// a launch (the stream then waits for the previous TMEM launch if that was on
// another stream), call launched() right after it; held for the launch.
class TmemOrder {
  public:
    explicit TmemOrder(cudaStream_t st);
    cudaError_t error() const { return err_; }
    cudaError_t launched();

  private:
    cudaStream_t st_;
    std::lock_guard<std::mutex> lock_;
    cudaError_t err_ = cudaSuccess;
    bool skip_ = false;
    int dev_ = 0;
};
// one bounded device wait driven into a configuration that cannot complete
cudaError_t wait_probe(int kind, int G, unsigned long long* words, unsigned int* ctr, int* err, long long limit,
                       cudaStream_t st);
// FP16 coarse operator with a per-(X, d) block scale, for the FP16-storage mode
void coarse_pack16(__half2* A16, float* s16, const double2* A, int nc, int Vc, cudaStream_t st);

// ---------------------------------------------------------------- batched (multi-RHS) coarse level
// Panel layout xB[X][b][n], n < npad (multiple of 16), complex FP32.
// Aemb: per (X, d) the 2nc x 2nc real embedding of A[X][d] in FP16, tensor-core layout.
void coarse_embed(__half* Aemb, const double2* A, int nc, int Vc, cudaStream_t st);
struct TcApplyArgs {
    const __half* Aemb;
    const float2* x;
    float2* y;
    int nc;
    int npad;
    int nw;         // panel columns per CTA (multiple of 16 dividing npad; 0: all)
    int dag;
    Geom g;
    float* norms;   // optional per-aggregate column sums of |y|^2: [Vc][npad]
    int* err;       // set to 1 if a bounded wait gave up
    const double* colscale;   // optional per-column power-of-two factor applied to x before the
                              // FP16 hi/lo split (y is scaled back exactly); nullptr: 1
    __half* bt;     // scratch for the split operand panel: tc_split_bytes(nc, npad) bytes
    int stages;     // pipeline stages per CTA (2 or 3; 0: as many as fit, up to 3)
};
// bytes of the FP16 hi/lo operand tiles of one panel (any chunk width)
inline size_t tc_split_bytes(int nc, int npad, long long Vc) { return (size_t)Vc * npad * (2 * nc) * 2 * sizeof(__half); }
// y = D_c x (dag: sigma3 D_c sigma3 x) for the whole panel on tcgen05 tensor cores;
// coarse_apply_tc_prepare(nc, npad) once per shape before launching (and before any capture)
bool coarse_apply_tc_supported(int nc, int npad);
cudaError_t coarse_apply_tc_prepare(int nc, int npad);
cudaError_t coarse_apply_tc(const TcApplyArgs& args, cudaStream_t st);
// autotuner: fastest chunk width (returned) and pipeline depth (*stages) for
// args' (nc, npad), timed once and cached
int coarse_apply_tc_tune(const TcApplyArgs& args, cudaStream_t st, int* stages);
// kernels launched by one bcg_iteration
constexpr int kBcgKernelsPerIteration = 10;   // two stencils of two launches each + six
// SIMT reference of the same contraction with the FP64 operator
template <typename T>
void coarse_apply_batched_simt(v2<T>* y, const double2* A, const v2<T>* x, int nc, int npad, bool dag, const Geom& g,
                               cudaStream_t st);

struct BatchScal {   // per-RHS CG scalars, npad doubles each
    double* scale;
    double* done;
    double* iters;
    double* r2;
    double* gamma;
    double* alpha;
    double* beta;
    double* csp;     // power-of-two panel scales of p and r for the FP16 split (from |s|^2, |r|^2)
    double* csr;
};
struct BatchCg {
    const __half* Aemb;
    __half* bt;      // split operand tiles of the stencil (scratch)
    int stages;      // pipeline depth of the stencil (from the autotuner)
    float2* y;
    float2* r;
    float2* s;
    float2* p;
    float2* q;
    const float2* rc;
    int nc, npad, nw, nrhs, maxit;
    double tol2;
    Geom g;
    BatchScal S;
    float* xpart;    // [Vc][npad]
    float* rpart;    // [kBatchRowChunks][npad]
    int* active;     // columns still iterating after the last check
    int* err;
};
constexpr int kBatchRowChunks = 1216;   // row chunks of the batched CG's column sums (8 per SM: enough warps to stream the panel)
void bcg_start(const BatchCg& c, cudaStream_t st);
void bcg_iteration(const BatchCg& c, cudaStream_t st);
void bcg_finish(const BatchCg& c, cudaStream_t st);
// nrhs stacked FP64 coarse vectors in[n][row] <-> panel [row][npad]
void panel_pack(float2* out, const double2* in, long long rows, int nrhs, int npad, cudaStream_t st);
void panel_unpack(double2* out, const float2* in, long long rows, int nrhs, int npad, cudaStream_t st);
void panel_pack64(double2* out, const double2* in, long long rows, int nrhs, int npad, cudaStream_t st);
void panel_unpack64(double2* out, const double2* in, long long rows, int nrhs, int npad, cudaStream_t st);

}  // namespace wmg

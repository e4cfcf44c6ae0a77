// Red-black (even-odd) preconditioned CG on the normal equations: the
// comparison solver of Sec. IV (Fig. 1 counts its Wilson matrix-vector
// products against MG-GCR, Fig. 2 its flops).
//
// With D = (4+m) I - H (eq. 2) and H coupling only opposite parities
// ((x+y+z+t) mod 2) on a lattice of even extents, the odd sites are
// eliminated:  Dhat = (4+m) - H_eo H_oe / (4+m) on the even sites,
// Dhat x_e = b_e + H_eo b_o / (4+m),  x_o = (b_o + H_oe x_e) / (4+m), and
// Dhat^dag = gamma5 Dhat gamma5.
//
// Layout (this solver only): checkerboarded SoA.  Parity p holds Vh = V/2
// sites, site (x,y,z,t) at cb index i = lex >> 1; a full vector is
// T2 v[p 2][k 12][Vh] (even half first), an even vector T2 v[k 12][Vh].
// Links per parity, the link U^mu_x stored at its site x: FP64
// double2 U[p][mu][e 9][Vh]; FP32 paired like the main dslash, float4
// U4[p][mu][j 4][Vh] (entries 2j, 2j+1) then float2 U8[p][mu][Vh] (entry 8).
// One thread per output site; consecutive threads read consecutive cb
// indices of every component.
#include "mg_launch.h"
#include "mg_wilson.cuh"

namespace wmg {

constexpr int kEoThreads = 256;

__host__ __device__ inline void eo_coords(const EoGeom& e, int p, long long i, int c[4]) {
    long long r = i / e.Lh0;
    const int xh = (int)(i - r * e.Lh0);
    c[1] = (int)(r % e.L[1]);
    r /= e.L[1];
    c[2] = (int)(r % e.L[2]);
    c[3] = (int)(r / e.L[2]);
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}
__host__ __device__ inline long long eo_lex(const EoGeom& e, const int c[4]) {
    return c[0] + (long long)e.L[0] * (c[1] + (long long)e.L[1] * (c[2] + (long long)e.L[2] * c[3]));
}

// ---------------------------------------------------------------- layout conversion
// boundary double2 [lex][12] <-> checkerboard T2 [p][12][Vh]
template <typename T>
__global__ void k_eo_spinor_pack(v2<T>* __restrict__ out, const double2* __restrict__ in, EoGeom e) {
    const long long V = 2 * e.Vh;
    long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= V) return;
    long long r = lex;
    int c[4];
    for (int m = 0; m < 4; ++m) { c[m] = (int)(r % e.L[m]); r /= e.L[m]; }
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    const long long i = lex >> 1;
    v2<T>* o = out + (size_t)p * 12 * e.Vh + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 v = in[lex * 12 + k];
        v2<T> w; w.x = (T)v.x; w.y = (T)v.y;
        o[(size_t)k * e.Vh] = w;
    }
}
template <typename T>
__global__ void k_eo_spinor_unpack(double2* __restrict__ out, const v2<T>* __restrict__ in, EoGeom e) {
    const long long V = 2 * e.Vh;
    long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= V) return;
    long long r = lex;
    int c[4];
    for (int m = 0; m < 4; ++m) { c[m] = (int)(r % e.L[m]); r /= e.L[m]; }
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    const v2<T>* s = in + (size_t)p * 12 * e.Vh + (lex >> 1);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const v2<T> v = s[(size_t)k * e.Vh];
        out[lex * 12 + k] = make_double2((double)v.x, (double)v.y);
    }
}
// internal FP64 links U[mu][X][9][l] -> U64[p][mu][9][Vh] and the paired FP32 copy
__global__ void k_eo_links_pack(double2* __restrict__ U64, float2* __restrict__ U32, const double2* __restrict__ Uint,
                                Geom g, EoGeom e) {
    long long sidx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (sidx >= g.V) return;
    const int X = (int)(sidx / g.Vb), l = (int)(sidx - (long long)X * g.Vb);
    const long long lex = lex_site(g, X, l);
    long long r = lex;
    int c[4];
    for (int m = 0; m < 4; ++m) { c[m] = (int)(r % e.L[m]); r /= e.L[m]; }
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    const long long i = lex >> 1;
    float4* u4 = reinterpret_cast<float4*>(U32);
    float2* u8 = U32 + (size_t)2 * 4 * 4 * e.Vh * 2;
    for (int mu = 0; mu < 4; ++mu) {
        double2 q[9];
        for (int k = 0; k < 9; ++k) q[k] = Uint[(((size_t)mu * g.Vc + X) * 9 + k) * g.Vb + l];
        const size_t pm = (size_t)p * 4 + mu;
        for (int k = 0; k < 9; ++k) U64[(pm * 9 + k) * e.Vh + i] = q[k];
        for (int j = 0; j < 4; ++j)
            u4[(pm * 4 + j) * e.Vh + i] = make_float4((float)q[2 * j].x, (float)q[2 * j].y, (float)q[2 * j + 1].x,
                                                      (float)q[2 * j + 1].y);
        u8[pm * e.Vh + i] = make_float2((float)q[8].x, (float)q[8].y);
    }
}

// ---------------------------------------------------------------- the half-lattice hop
template <typename T>
__device__ __forceinline__ void eo_link(cx<T> (&m)[9], const void* U, const EoGeom& e, int p, int mu, long long i) {
    const size_t pm = (size_t)p * 4 + mu;
    if constexpr (sizeof(T) == 4) {
        const float4* u4 = reinterpret_cast<const float4*>(U) + pm * 4 * e.Vh + i;
        const float2* u8 = reinterpret_cast<const float2*>(U) + (size_t)2 * 4 * 4 * e.Vh * 2 + pm * e.Vh + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 q = __ldg(u4 + (size_t)j * e.Vh);
            m[2 * j] = cx<T>(q.x, q.y);
            m[2 * j + 1] = cx<T>(q.z, q.w);
        }
        const float2 q8 = __ldg(u8);
        m[8] = cx<T>(q8.x, q8.y);
    } else {
        const v2<T>* u = reinterpret_cast<const v2<T>*>(U) + pm * 9 * e.Vh + i;
#pragma unroll
        for (int q = 0; q < 9; ++q) m[q] = ldg<T>(u + (size_t)q * e.Vh);
    }
}

// acc += (1 -/+ gamma_mu)/2 W psi(y) for the neighbour y of x in +-mu (the H of eq. 2)
template <typename T, int MU, bool FWD, bool G5IN>
__device__ __forceinline__ void eo_hop1(cx<T> (&acc)[4][3], const v2<T>* __restrict__ in, const void* U,
                                        const EoGeom& e, int p, long long i, const int (&c)[4]) {
    int cn[4] = {c[0], c[1], c[2], c[3]};
    bool flip = false;
    cn[MU] += FWD ? 1 : -1;
    if (cn[MU] == e.L[MU]) { cn[MU] = 0; flip = (MU == 3) && e.tap; }
    if (cn[MU] < 0) { cn[MU] = e.L[MU] - 1; flip = (MU == 3) && e.tap; }
    const long long j = eo_lex(e, cn) >> 1;
    cx<T> ps[4][3];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<T> v = ldg<T>(in + (size_t)(3 * s + a) * e.Vh + j);
            ps[s][a] = (G5IN && s >= 2) ? cx<T>(-v.r, -v.i) : v;
        }
    cx<T> h[2][3];
    project<T, MU, FWD>(ps, h);
    cx<T> m[9];
    if (FWD) eo_link<T>(m, U, e, p, MU, i);          // U^mu_x, stored at x (parity p)
    else eo_link<T>(m, U, e, 1 - p, MU, j);          // U^mu_{x-mu}, stored at x - mu (parity 1 - p)
    cx<T> w[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) { w[0][a] = cx<T>(0, 0); w[1][a] = cx<T>(0, 0); }
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
    accumulate<T, MU, FWD>(acc, w, flip ? T(-0.5) : T(0.5));
}

// out_p = c_src src + c_self self + c_h G (H in) [+ out if EO_ACC], for the sites
// of parity p (in: parity 1 - p; src, self, out: parity p, each an even-sized
// [12][Vh] array), G = gamma5 when EO_G5H; EO_G5IN reads gamma5 in; EO_NORM
// writes |out|^2 (grid-reduced) to R.scal[slot]; EO_SKIP: nothing to do once
// R.scal[done_slot] is set (the CG has converged).
template <typename T, int F>
__global__ void __launch_bounds__(kEoThreads) k_eo_hop(v2<T>* __restrict__ out, const v2<T>* __restrict__ in,
                                                       const v2<T>* __restrict__ src, const v2<T>* __restrict__ self,
                                                       const void* __restrict__ U, EoGeom e, int p, T c_src, T c_self,
                                                       T c_h, int slot, int done_slot, Reduce R) {
    if ((F & EO_SKIP) && R.scal[done_slot] != 0.0) return;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    T nrm = 0;
    if (i < e.Vh) {
        int c[4];
        eo_coords(e, p, i, c);
        cx<T> acc[4][3];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[s][a] = cx<T>(0, 0);
        constexpr bool G5 = (F & EO_G5IN) != 0;
        eo_hop1<T, 0, true, G5>(acc, in, U, e, p, i, c);
        eo_hop1<T, 0, false, G5>(acc, in, U, e, p, i, c);
        eo_hop1<T, 1, true, G5>(acc, in, U, e, p, i, c);
        eo_hop1<T, 1, false, G5>(acc, in, U, e, p, i, c);
        eo_hop1<T, 2, true, G5>(acc, in, U, e, p, i, c);
        eo_hop1<T, 2, false, G5>(acc, in, U, e, p, i, c);
        eo_hop1<T, 3, true, G5>(acc, in, U, e, p, i, c);
        eo_hop1<T, 3, false, G5>(acc, in, U, e, p, i, c);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const size_t k = (size_t)(3 * s + a) * e.Vh + i;
                cx<T> h = acc[s][a];
                if ((F & EO_G5H) && s >= 2) h = cx<T>(-h.r, -h.i);
                cx<T> v = c_h * h;
                if (F & EO_SRC) v = v + c_src * ld<T>(src + k);
                if (F & EO_SELF) v = v + c_self * ld<T>(self + k);
                if (F & EO_ACC) v = v + ld<T>(out + k);
                st<T>(out + k, v);
                if (F & EO_NORM) nrm += norm2(v);
            }
    }
    if (F & EO_NORM) {
        T v1[1] = {nrm};
        grid_reduce<1, T>(v1, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) { R.scal[slot] = t[0]; });
    }
}

static inline int eo_grid(long long n) { return (int)((n + kEoThreads - 1) / kEoThreads); }

template <typename T>
void eo_hop(int flags, v2<T>* out, const v2<T>* in, const v2<T>* src, const v2<T>* self, const void* U,
            const EoGeom& e, int p, double c_src, double c_self, double c_h, int slot, int done_slot, const Reduce& R,
            cudaStream_t st) {
    const int grid = eo_grid(e.Vh);
#define EO_CASE(FL)                                                                                            \
    case FL:                                                                                                   \
        note_launch();                                                                                         \
        k_eo_hop<T, FL><<<grid, kEoThreads, 0, st>>>(out, in, src, self, U, e, p, (T)c_src, (T)c_self, (T)c_h, \
                                                     slot, done_slot, R);                                      \
        break;
    switch (flags) {
        EO_CASE(EO_PLAIN)
        EO_CASE(EO_G5IN)
        EO_CASE(EO_SKIP)
        EO_CASE(EO_SKIP | EO_G5IN)
        EO_CASE(EO_SKIP | EO_SELF | EO_NORM)
        EO_CASE(EO_SKIP | EO_SELF | EO_NORM | EO_G5H)
        EO_CASE(EO_SELF | EO_NORM)
        EO_CASE(EO_SELF | EO_NORM | EO_G5H)
        EO_CASE(EO_SRC | EO_SELF | EO_NORM)
        EO_CASE(EO_SRC)
        EO_CASE(EO_SRC | EO_ACC)
        default: break;
    }
#undef EO_CASE
}
template void eo_hop<float>(int, v2<float>*, const v2<float>*, const v2<float>*, const v2<float>*, const void*,
                            const EoGeom&, int, double, double, double, int, int, const Reduce&, cudaStream_t);
template void eo_hop<double>(int, v2<double>*, const v2<double>*, const v2<double>*, const v2<double>*, const void*,
                             const EoGeom&, int, double, double, double, int, int, const Reduce&, cudaStream_t);

// ---------------------------------------------------------------- CGLS steps (device scalars)
// x += alpha p, r -= alpha q with alpha = gamma / |q|^2; |r|^2 -> scal[r2_slot];
// |r|^2 <= tol2 marks the solve done and records the iteration count.
template <typename T>
__global__ void __launch_bounds__(kEoThreads) k_eo_cg_update1(v2<T>* __restrict__ x, v2<T>* __restrict__ r,
                                                              const v2<T>* __restrict__ p, const v2<T>* __restrict__ q,
                                                              long long n, EoCgSlots s, int iter, Reduce R) {
    if (R.scal[s.done] != 0.0) return;
    const double qq = R.scal[s.q2];
    const T alpha = qq > 0 ? (T)(R.scal[s.gamma] / qq) : T(0);
    T acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        cx<T> xv = ld<T>(x + i), rv = ld<T>(r + i);
        const cx<T> pv = ld<T>(p + i), qv = ld<T>(q + i);
        xv = xv + alpha * pv;
        rv = rv - alpha * qv;
        st<T>(x + i, xv);
        st<T>(r + i, rv);
        acc += norm2(rv);
    }
    T v1[1] = {acc};
    grid_reduce<1, T>(v1, R.partials, R.ticket, R.partial_bytes, [&](double (&t)[1]) {
        R.scal[s.r2] = t[0];
        R.scal[s.iters] = (double)(iter + 1);
        if (t[0] <= R.scal[s.tol2] || !(qq > 0)) R.scal[s.done] = 1.0;
    });
}
// p = s + beta p, beta = |s|^2 / gamma_old; then gamma = |s|^2 (the new value
// lives in its own slot: gamma slots alternate with the iteration parity)
template <typename T>
__global__ void __launch_bounds__(kEoThreads) k_eo_cg_update2(v2<T>* __restrict__ p, const v2<T>* __restrict__ sv,
                                                              long long n, int gamma_old, int gamma_new, int done,
                                                              Reduce R) {
    if (R.scal[done] != 0.0) return;
    const double g0 = R.scal[gamma_old];
    const T beta = g0 > 0 ? (T)(R.scal[gamma_new] / g0) : T(0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        st<T>(p + i, ld<T>(sv + i) + beta * ld<T>(p + i));
}
template <typename T>
void eo_cg_update1(v2<T>* x, v2<T>* r, const v2<T>* p, const v2<T>* q, long long n, const EoCgSlots& s, int iter,
                   const Reduce& R, cudaStream_t st) {
    long long b = (n + kEoThreads - 1) / kEoThreads;
    if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
    note_launch();
    k_eo_cg_update1<T><<<(int)b, kEoThreads, 0, st>>>(x, r, p, q, n, s, iter, R);
}
template <typename T>
void eo_cg_update2(v2<T>* p, const v2<T>* sv, long long n, int gamma_old, int gamma_new, int done, const Reduce& R,
                   cudaStream_t st) {
    long long b = (n + kEoThreads - 1) / kEoThreads;
    if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
    note_launch();
    k_eo_cg_update2<T><<<(int)b, kEoThreads, 0, st>>>(p, sv, n, gamma_old, gamma_new, done, R);
}
template void eo_cg_update1<float>(v2<float>*, v2<float>*, const v2<float>*, const v2<float>*, long long,
                                   const EoCgSlots&, int, const Reduce&, cudaStream_t);
template void eo_cg_update1<double>(v2<double>*, v2<double>*, const v2<double>*, const v2<double>*, long long,
                                    const EoCgSlots&, int, const Reduce&, cudaStream_t);
template void eo_cg_update2<float>(v2<float>*, const v2<float>*, long long, int, int, int, const Reduce&, cudaStream_t);
template void eo_cg_update2<double>(v2<double>*, const v2<double>*, long long, int, int, int, const Reduce&,
                                    cudaStream_t);

template <typename T> void eo_spinor_pack(v2<T>* out, const double2* in, const EoGeom& e, cudaStream_t st) {
    note_launch();
    k_eo_spinor_pack<T><<<eo_grid(2 * e.Vh), kEoThreads, 0, st>>>(out, in, e);
}
template <typename T> void eo_spinor_unpack(double2* out, const v2<T>* in, const EoGeom& e, cudaStream_t st) {
    note_launch();
    k_eo_spinor_unpack<T><<<eo_grid(2 * e.Vh), kEoThreads, 0, st>>>(out, in, e);
}
template void eo_spinor_pack<float>(v2<float>*, const double2*, const EoGeom&, cudaStream_t);
template void eo_spinor_pack<double>(v2<double>*, const double2*, const EoGeom&, cudaStream_t);
template void eo_spinor_unpack<float>(double2*, const v2<float>*, const EoGeom&, cudaStream_t);
template void eo_spinor_unpack<double>(double2*, const v2<double>*, const EoGeom&, cudaStream_t);
void eo_links_pack(double2* U64, float2* U32, const double2* Uint, const Geom& g, const EoGeom& e, cudaStream_t st) {
    note_launch();
    k_eo_links_pack<<<eo_grid(g.V), kEoThreads, 0, st>>>(U64, U32, Uint, g, e);
}

}  // namespace wmg

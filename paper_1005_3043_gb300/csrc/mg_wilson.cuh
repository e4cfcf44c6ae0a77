// Spin projection and reconstruction of the Wilson hop (eq. 2) in the
// DeGrand-Rossi basis, shared by the dslash kernels of every storage precision.
#pragma once
#include "mg_common.cuh"

namespace wmg {

// Spin projection in the DeGrand-Rossi basis.  FWD: (1 - gamma_mu) psi(x+mu);
// BWD: (1 + gamma_mu) psi(x-mu).  Both are rank-2 projectors: the upper two
// spin components h0, h1 determine the lower two.
template <typename T, int MU, bool FWD>
__device__ __forceinline__ void project(const cx<T> (&p)[4][3], cx<T> (&h)[2][3]) {
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
}
// acc += coef * reconstruct(w): components 0,1 are w0, w1; 2,3 follow from the projector
template <typename T, int MU, bool FWD>
__device__ __forceinline__ void accumulate(cx<T> (&acc)[4][3], const cx<T> (&w)[2][3], T coef) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<T> w0 = coef * w[0][c], w1 = coef * w[1][c];
        acc[0][c] = acc[0][c] + w0;
        acc[1][c] = acc[1][c] + w1;
        if (MU == 0) {
            acc[2][c] = acc[2][c] + (FWD ? mul_i(w1) : mul_mi(w1));
            acc[3][c] = acc[3][c] + (FWD ? mul_i(w0) : mul_mi(w0));
        } else if (MU == 1) {
            acc[2][c] = FWD ? acc[2][c] - w1 : acc[2][c] + w1;
            acc[3][c] = FWD ? acc[3][c] + w0 : acc[3][c] - w0;
        } else if (MU == 2) {
            acc[2][c] = acc[2][c] + (FWD ? mul_i(w0) : mul_mi(w0));
            acc[3][c] = acc[3][c] + (FWD ? mul_mi(w1) : mul_i(w1));
        } else {
            acc[2][c] = FWD ? acc[2][c] - w0 : acc[2][c] + w0;
            acc[3][c] = FWD ? acc[3][c] - w1 : acc[3][c] + w1;
        }
    }
}

}  // namespace wmg

// Geometry of axis-aligned box cells and faces, shared by the assembly and
// the adjoint kernels.  ref holds the reference-element matrices built by
// k_ref_matrices: [0..2] (2-D) or [0..5] (3-D) cell blocks of 144 entries,
// [6] the 2-D edge masses, [6..7] the 3-D face-mass blocks (4x4, stride 4).
#pragma once

#include "common.cuh"

namespace thm {

__device__ __forceinline__ double vdist(const double* X, int dim, int64_t p, int64_t q) {
    double s = 0;
    for (int k = 0; k < dim; ++k) {
        double t = X[q * dim + k] - X[p * dim + k];
        s += t * t;
    }
    return sqrt(s);
}

// Side lengths of a box cell along its local axes xi (v0->v1), eta (v0->v2), zeta (v0->v4).
__device__ __forceinline__ void cell_sides(const double* X, int dim, const int32_t* cells, int64_t c, double* h) {
    const int nv = dim == 2 ? 4 : 8;
    const int32_t* cv = cells + c * nv;
    h[0] = vdist(X, dim, cv[0], cv[1]);
    h[1] = vdist(X, dim, cv[0], cv[2]);
    h[2] = dim == 3 ? vdist(X, dim, cv[0], cv[4]) : 1.0;
}

// Local curl-curl and mass entries (kr, kc) of a box cell (unsigned, local basis).
// 2-D: A = ref0/(ab), M = (b/a) ref1 + (a/b) ref2.
// 3-D: A = sum_k h_k^2/(abc) ref_k, M = sum_k abc/h_k^2 ref_{3+k}.
__device__ __forceinline__ void cell_am(int dim, const double* ref, int nb, const double* h, int kr, int kc,
                                        double& A, double& M) {
    const int o = kr * nb + kc;
    if (dim == 2) {
        const double a = h[0], b = h[1];
        A = ref[o] / (a * b);
        M = (b / a) * ref[144 + o] + (a / b) * ref[288 + o];
        return;
    }
    const double V = h[0] * h[1] * h[2];
    A = 0;
    M = 0;
    for (int k = 0; k < 3; ++k) {
        A += h[k] * h[k] / V * ref[k * 144 + o];
        M += V / (h[k] * h[k]) * ref[(3 + k) * 144 + o];
    }
}

// Local entry (kr, kc) of a cell: mu^{-1} A - omega^2 M.
__device__ __forceinline__ double cell_entry(int dim, const double* ref, int nb, double mu, double w2,
                                             const double* h, int kr, int kc) {
    double A, M;
    cell_am(dim, ref, nb, h, kr, kc, A, M);
    return mu * A - w2 * M;
}

// Tangential mass of face f between its local DOFs a and b (unsigned).
__device__ __forceinline__ double face_mass(int dim, const double* ref, const double* X, const int32_t* fv, int a,
                                            int b) {
    if (dim == 2) {
        if (a != b) return 0.0;                   // Whitney and gradient traces are L2-orthogonal
        return ref[6 * 144 + a] / vdist(X, 2, fv[0], fv[1]);
    }
    const double p = vdist(X, 3, fv[0], fv[1]), q = vdist(X, 3, fv[0], fv[2]);
    return (q / p) * ref[6 * 144 + a * 4 + b] + (p / q) * ref[7 * 144 + a * 4 + b];
}


}  // namespace thm

// Assembly of the subdomain operators T_i = P_i + i B_i (Section 2, the
// integrals (A), (M), (B) and Eq. 3; Section 3.1, the transmission term of
// Eq. 5), the Dirichlet data and lifting, and the factorisation of the block
// preconditioner P_i = A_i - omega^2 M_i of Eq. 7.
#include <cmath>

#include "common.cuh"
#include "element.cuh"

namespace thm {

// ---------------------------------------------------------------------------
// Reference matrices.  Every component of a reference basis function (and of
// its curl) is c * f(xi) * g(eta) with f, g from five quadratics; integrals of
// products of two such terms are exact sums of monomial integrals 1/(i+j+1).
// Output layout: ref[0] = int curl_i curl_j, ref[1] = int phi_i,x phi_j,x,
// ref[2] = int phi_i,y phi_j,y on the unit square (12 x 12 each, row-major).
// Per cell of sides a (xi) and b (eta):  A = ref0/(ab),  M = (b/a) ref1 + (a/b) ref2.
// ---------------------------------------------------------------------------
__constant__ double c_poly[5][3] = {
    {1, 0, 0},     // 1
    {0, 1, 0},     // t
    {1, -1, 0},    // 1 - t
    {0, 1, -1},    // q(t)  = t (1 - t)
    {1, -2, 0},    // q'(t) = 1 - 2t
};

struct Term {
    double c;
    int f, g, h;      // 1-D factors in xi, eta, zeta (h = 0: the constant, for 2-D)
};

// Terms (x component, y component, curl) of the 12 order-2 functions in the
// local order [W0 G0 W1 G1 W2 G2 W3 G3 B0 B1 B2 B3]; order 1 uses W0..W3.
__device__ void basis_terms(int order, int i, Term& x, Term& y, Term& cu) {
    const Term Z{0, 0, 0, 0};
    // Whitney functions of local edges 0..3
    const Term Wx[4] = {{1, 0, 2}, {1, 0, 1}, Z, Z};
    const Term Wy[4] = {Z, Z, {1, 2, 0}, {1, 1, 0}};
    const Term Wc[4] = {{1, 0, 0}, {-1, 0, 0}, {-1, 0, 0}, {1, 0, 0}};
    // gradient functions grad(q(s) * ramp)
    const Term Gx[4] = {{1, 4, 2}, {1, 4, 1}, {-1, 0, 3}, {1, 0, 3}};
    const Term Gy[4] = {{-1, 3, 0}, {1, 3, 0}, {1, 2, 4}, {1, 1, 4}};
    // cell bubbles
    const Term Bx[4] = {{1, 2, 3}, {1, 1, 3}, Z, Z};
    const Term By[4] = {Z, Z, {1, 3, 2}, {1, 3, 1}};
    const Term Bc[4] = {{-1, 2, 4}, {-1, 1, 4}, {1, 4, 2}, {1, 4, 1}};
    if (order == 1) {
        x = Wx[i]; y = Wy[i]; cu = Wc[i];
        return;
    }
    if (i < 8) {
        int k = i >> 1;
        if ((i & 1) == 0) { x = Wx[k]; y = Wy[k]; cu = Wc[k]; }
        else { x = Gx[k]; y = Gy[k]; cu = Z; }
    } else {
        int k = i - 8;
        x = Bx[k]; y = By[k]; cu = Bc[k];
    }
}

__device__ double int1(int f, int g) {
    double s = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (c_poly[f][i] != 0 && c_poly[g][j] != 0) s += c_poly[f][i] * c_poly[g][j] / (double)(i + j + 1);
    return s;
}

__device__ double int2(const Term& a, const Term& b) {
    if (a.c == 0 || b.c == 0) return 0.0;
    return a.c * b.c * int1(a.f, b.f) * int1(a.g, b.g) * int1(a.h, b.h);
}

// Order-1 hex: 12 Whitney functions in the local edge order (xi-edges at
// (eta,zeta) = 00,10,01,11, then eta-edges at (xi,zeta), then zeta-edges at
// (xi,eta)); comp[3] = value components, cu[3] = reference curl components.
// L(t;0) = 1 - t (poly 2), L(t;1) = t (poly 1), dL(0) = -1, dL(1) = +1.
__device__ void basis_terms3(int i, Term* comp, Term* cu) {
    const Term Z{0, 0, 0, 0};
    const int ax = i / 4, e0 = (i % 4) & 1, e1 = (i % 4) >> 1;
    const int L0 = e0 ? 1 : 2, L1 = e1 ? 1 : 2;
    const double d0 = e0 ? 1.0 : -1.0, d1 = e1 ? 1.0 : -1.0;
    for (int k = 0; k < 3; ++k) { comp[k] = Z; cu[k] = Z; }
    if (ax == 0) {           // (L(eta) L(zeta), 0, 0); curl = (0, L(eta) dL(zeta), -dL(eta) L(zeta))
        comp[0] = Term{1, 0, L0, L1};
        cu[1] = Term{d1, 0, L0, 0};
        cu[2] = Term{-d0, 0, 0, L1};
    } else if (ax == 1) {    // (0, L(xi) L(zeta), 0); curl = (-L(xi) dL(zeta), 0, dL(xi) L(zeta))
        comp[1] = Term{1, L0, 0, L1};
        cu[0] = Term{-d1, L0, 0, 0};
        cu[2] = Term{d0, 0, 0, L1};
    } else {                 // (0, 0, L(xi) L(eta)); curl = (L(xi) dL(eta), -dL(xi) L(eta), 0)
        comp[2] = Term{1, L0, L1, 0};
        cu[0] = Term{d1, L0, 0, 0};
        cu[1] = Term{-d0, 0, L1, 0};
    }
}

// ref layout (144 doubles per matrix, row stride nb):
//  2-D: [0] int curl curl, [1] int phi_x phi_x, [2] int phi_y phi_y,
//       [6] face (edge) scalars: [0] int 1*1, [1] int q'(s)^2
//  3-D: [0..2] int curl_a curl_a (a = xi, eta, zeta), [3..5] int phi_a phi_a,
//       [6], [7] the order-1 quad face mass parts (row stride 4)
__global__ void k_ref_matrices(int dim, int order, int nb, double* ref) {
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        int i = t / nb, j = t % nb;
        if (j < i) continue;
        if (dim == 2) {
            Term xi, yi, ci, xj, yj, cj;
            basis_terms(order, i, xi, yi, ci);
            basis_terms(order, j, xj, yj, cj);
            double a = int2(ci, cj), mx = int2(xi, xj), my = int2(yi, yj);
            ref[0 * 144 + i * nb + j] = a;  ref[0 * 144 + j * nb + i] = a;
            ref[1 * 144 + i * nb + j] = mx; ref[1 * 144 + j * nb + i] = mx;
            ref[2 * 144 + i * nb + j] = my; ref[2 * 144 + j * nb + i] = my;
        } else {
            Term vi[3], ci[3], vj[3], cj[3];
            basis_terms3(i, vi, ci);
            basis_terms3(j, vj, cj);
            for (int k = 0; k < 3; ++k) {
                double aa = int2(ci[k], cj[k]), mm = int2(vi[k], vj[k]);
                ref[k * 144 + i * nb + j] = aa;       ref[k * 144 + j * nb + i] = aa;
                ref[(3 + k) * 144 + i * nb + j] = mm; ref[(3 + k) * 144 + j * nb + i] = mm;
            }
        }
    }
    if (threadIdx.x == 0) {
        if (dim == 2) {
            ref[6 * 144 + 0] = int1(0, 0);
            ref[6 * 144 + 1] = int1(4, 4);
        } else {
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    Term xi, yi, ci, xj, yj, cj;
                    basis_terms(1, i, xi, yi, ci);
                    basis_terms(1, j, xj, yj, cj);
                    ref[6 * 144 + i * 4 + j] = int2(xi, xj);
                    ref[7 * 144 + i * 4 + j] = int2(yi, yj);
                }
        }
    }
}

// Gather-by-row assembly of P_i in the SELL layout.  Entry (r, col) sums the
// cells holding both DOFs in ascending cell order; entry (col, r) visits the
// same cells in the same order with exactly symmetric reference entries, so
// P_i is bit-symmetric.
__global__ void k_assemble(int dim, int64_t n_loc, int nb, int maxc, const double* __restrict__ ref,
                           const double* __restrict__ X, const int32_t* __restrict__ cells,
                           const int8_t* __restrict__ signs, const int32_t* __restrict__ cell_loc,
                           const double* __restrict__ mu, const double* __restrict__ w2c,
                           const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                           const uint8_t* __restrict__ pad, const int32_t* __restrict__ row_cell,
                           const int32_t* __restrict__ row_k, double* __restrict__ val64,
                           float* __restrict__ val32) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_loc) return;
    int64_t sl = r / SELL_C;
    int lane = (int)(r % SELL_C);
    int64_t base = slice_ptr[sl];
    int w = (int)((slice_ptr[sl + 1] - base) / SELL_C);
    for (int t = 0; t < w; ++t) {
        int64_t idx = base + (int64_t)t * SELL_C + lane;
        double v = 0.0;
        if (!pad[idx]) {
            int32_t cc = col[idx];
            for (int u = 0; u < maxc; ++u) {
                int32_t c = row_cell[r * maxc + u];
                if (c < 0) break;
                int kr = row_k[r * maxc + u];
                for (int kc = 0; kc < nb; ++kc) {
                    if (cell_loc[(int64_t)c * nb + kc] != cc) continue;
                    double hh[3];
                    cell_sides(X, dim, cells, c, hh);
                    double s = (double)(signs[(int64_t)c * nb + kr] * signs[(int64_t)c * nb + kc]);
                    v += s * cell_entry(dim, ref, nb, mu[c], w2c[c], hh, kr, kc);
                }
            }
        }
        val64[idx] = v;
        val32[idx] = (float)v;
    }
}

// Impedance / transmission face terms, gathered per local row from the faces
// whose terms reach it (kind 1: Gamma^inf, kind 2: Sigma), times kappa*omega.
// 2-D: the face mass is diagonal, stored per row (bg, bs).  3-D: the face mass
// couples the four edges of a face; stored on the SELL pattern (bvg, bvs).
__global__ void k_face_terms(int dim, int64_t n_loc, int fd, const double* __restrict__ ref,
                             const double* __restrict__ X, const int32_t* __restrict__ face_v,
                             const int8_t* __restrict__ face_sgn, const int8_t* __restrict__ face_kind,
                             const int32_t* __restrict__ face_loc, const int32_t* __restrict__ row_face,
                             const int8_t* __restrict__ row_face_a, const int8_t* __restrict__ row_face_side,
                             const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                             const uint8_t* __restrict__ pad, const double* __restrict__ kwf, double tre,
                             double tim, double* val64, float* val32, double* bg64,
                             double* bs64, float* bg32,
                             float* bs32, double* bvg64, double* bvs64, float* bvg32, float* bvs32) {
    // Sigma terms: (tre + i tim) kappa omega M_Sigma; the imaginary part goes to
    // the face-term arrays, a real part (tre != 0) into the values of P_i
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_loc) return;
    constexpr int RF = thm_mesh::RF;
    if (dim == 2) {
        double g = 0, s = 0;
        for (int u = 0; u < RF; ++u) {
            const int32_t f = row_face[r * RF + u];
            if (f < 0) continue;
            const int a = row_face_a[r * RF + u];
            const double v = kwf[f] * face_mass(2, ref, X, face_v + (int64_t)f * 4, a, a);
            if (face_kind[f] == 1) g += v; else s += v;
        }
        bg64[r] = g; bs64[r] = tim * s; bg32[r] = (float)g; bs32[r] = (float)(tim * s);
        if (tre != 0.0 && s != 0.0) {
            const int64_t sl = r / SELL_C;
            const int lane = (int)(r % SELL_C);
            const int64_t base = slice_ptr[sl];
            const int w = (int)((slice_ptr[sl + 1] - base) / SELL_C);
            for (int t = 0; t < w; ++t) {
                const int64_t idx = base + (int64_t)t * SELL_C + lane;
                if (!pad[idx] && col[idx] == r) {
                    val64[idx] += tre * s;
                    val32[idx] = (float)val64[idx];
                }
            }
        }
        return;
    }
    bg64[r] = 0; bs64[r] = 0; bg32[r] = 0; bs32[r] = 0;
    const int64_t sl = r / SELL_C;
    const int lane = (int)(r % SELL_C);
    const int64_t base = slice_ptr[sl];
    const int w = (int)((slice_ptr[sl + 1] - base) / SELL_C);
    for (int t = 0; t < w; ++t) {
        const int64_t idx = base + (int64_t)t * SELL_C + lane;
        double g = 0, s = 0;
        if (!pad[idx]) {
            const int32_t cc = col[idx];
            for (int u = 0; u < RF; ++u) {
                const int32_t f = row_face[r * RF + u];
                if (f < 0) continue;
                const int a = row_face_a[r * RF + u], side = row_face_side[r * RF + u];
                for (int b = 0; b < fd; ++b) {
                    if (face_loc[((int64_t)f * 2 + side) * fd + b] != cc) continue;
                    const double v = kwf[f] * face_sgn[(int64_t)f * fd + a] * face_sgn[(int64_t)f * fd + b] *
                                     face_mass(3, ref, X, face_v + (int64_t)f * 4, a, b);
                    if (face_kind[f] == 1) g += v; else s += v;
                }
            }
        }
        bvg64[idx] = g; bvs64[idx] = tim * s; bvg32[idx] = (float)g; bvs32[idx] = (float)(tim * s);
        if (tre != 0.0 && s != 0.0) {
            val64[idx] += tre * s;
            val32[idx] = (float)val64[idx];
        }
    }
}

// Values of the interface-entry terms: kappa*omega times the signed face mass
// between DOFs a and b.
__global__ void k_iface_vals(int dim, int64_t n_terms, int fd, const double* __restrict__ ref,
                             const double* __restrict__ X, const int32_t* __restrict__ face_v,
                             const int8_t* __restrict__ face_sgn, const int32_t* __restrict__ tf,
                             const int8_t* __restrict__ ta, const int8_t* __restrict__ tb,
                             const double* __restrict__ kwf, double* __restrict__ val) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n_terms) return;
    const int32_t f = tf[p];
    const int a = ta[p], b = tb[p];
    val[p] = kwf[f] * face_sgn[(int64_t)f * fd + a] * face_sgn[(int64_t)f * fd + b] *
             face_mass(dim, ref, X, face_v + (int64_t)f * 4, a, b);
}

// Dirichlet values: tangential moments of E^inc(x) = pol exp(-i omega dir.x)
// along the global direction lo -> hi, by 8-point Gauss-Legendre on [0,1]:
//   Whitney DOF  m0 = l int_0^1 E_t(s) ds,
//   gradient DOF m1 = 3 l int_0^1 E_t(s) (1 - 2s) ds.
__constant__ double c_gl8_x[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                                  -0.1834346424956498, 0.1834346424956498,  0.5255324099163290,
                                  0.7966664774136267,  0.9602898564975363};
__constant__ double c_gl8_w[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                                  0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                                  0.2223810344533745, 0.1012285362903763};

__global__ void k_dirichlet(int64_t n_de, int dim, int order, const int64_t* __restrict__ edges,
                            const double* __restrict__ X, const int64_t* __restrict__ elo,
                            const int64_t* __restrict__ ehi, const double* __restrict__ om, double pr0, double pi0,
                            double pr1, double pi1, double pr2, double pi2, double d0, double d1,
                            double d2, double2* __restrict__ uD) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_de) return;
    int64_t e = edges[t];
    double xl[3] = {0, 0, 0}, tv[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
        xl[k] = X[elo[e] * dim + k];
        tv[k] = X[ehi[e] * dim + k] - xl[k];
    }
    double l = sqrt(tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2]);
    // pol . t_hat
    double ptr = (pr0 * tv[0] + pr1 * tv[1] + pr2 * tv[2]) / l;
    double pti = (pi0 * tv[0] + pi1 * tv[1] + pi2 * tv[2]) / l;
    const double omega = om[t];
    double m0r = 0, m0i = 0, m1r = 0, m1i = 0;
    for (int q = 0; q < 8; ++q) {
        double s = 0.5 * (c_gl8_x[q] + 1.0), wq = 0.5 * c_gl8_w[q];
        double ph = -omega * (d0 * (xl[0] + s * tv[0]) + d1 * (xl[1] + s * tv[1]) + d2 * (xl[2] + s * tv[2]));
        double sn, cs;
        sincos(ph, &sn, &cs);
        double er = ptr * cs - pti * sn, ei = ptr * sn + pti * cs;
        m0r += wq * er; m0i += wq * ei;
        m1r += wq * er * (1.0 - 2.0 * s); m1i += wq * ei * (1.0 - 2.0 * s);
    }
    if (order == 1) {
        uD[e] = make_double2(l * m0r, l * m0i);
    } else {
        uD[2 * e] = make_double2(l * m0r, l * m0i);
        uD[2 * e + 1] = make_double2(3.0 * l * m1r, 3.0 * l * m1i);
    }
}

// Dirichlet values given by the caller: u_D[ids[t]] = vals[t].
__global__ void k_dirichlet_given(int64_t n_dir, const int64_t* __restrict__ ids, const double2* __restrict__ vals,
                                  double2* __restrict__ uD) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n_dir) uD[ids[t]] = vals[t];
}

// Lifting: f_i = -(P_i)_{F,D} u_D from the cells of each row (2-D: the face
// terms never couple a free DOF to a Dirichlet one).
__global__ void k_lifting(int dim, int64_t n_loc, int nb, int maxc, const double* __restrict__ ref,
                          const double* __restrict__ X, const int32_t* __restrict__ cells,
                          const int8_t* __restrict__ signs, const int32_t* __restrict__ cell_loc,
                          const int32_t* __restrict__ cell_dofs, const double* __restrict__ mu,
                          const double* __restrict__ w2c,
                          const int32_t* __restrict__ row_cell, const int32_t* __restrict__ row_k,
                          const double2* __restrict__ uD, int fd, const int32_t* __restrict__ face_v,
                          const int32_t* __restrict__ face_dof, const int8_t* __restrict__ face_sgn,
                          const int32_t* __restrict__ face_loc, const int32_t* __restrict__ row_face,
                          const int8_t* __restrict__ row_face_a, const int8_t* __restrict__ row_face_side,
                          const int8_t* __restrict__ face_kind, const double* __restrict__ kwf, double tre,
                          double tim, double2* __restrict__ f,
                          double2* __restrict__ fres) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_loc) return;
    double fr = 0, fi = 0;
    for (int u = 0; u < maxc; ++u) {
        int32_t c = row_cell[r * maxc + u];
        if (c < 0) break;
        int kr = row_k[r * maxc + u];
        double hh[3];
        cell_sides(X, dim, cells, c, hh);
        for (int kc = 0; kc < nb; ++kc) {
            if (cell_loc[(int64_t)c * nb + kc] >= 0) continue;
            double s = (double)(signs[(int64_t)c * nb + kr] * signs[(int64_t)c * nb + kc]);
            double v = s * cell_entry(dim, ref, nb, mu[c], w2c[c], hh, kr, kc);
            double2 d = uD[cell_dofs[(int64_t)c * nb + kc]];
            fr -= v * d.x;
            fi -= v * d.y;
        }
    }
    // face terms coupling the row to Dirichlet DOFs: -(i kappa omega M_f) u_D.
    // The global system holds only the Gamma^inf faces; the subdomain operator
    // T_i also the transmission faces of Sigma, with the coefficient
    // (tre + i tim) kappa omega (3-D only: in 2-D no Dirichlet DOF lies on an
    // interface edge).
    double gr = fr, gi = fi;
    constexpr int RF = thm_mesh::RF;
    for (int u = 0; u < RF; ++u) {
        const int32_t f = row_face[r * RF + u];
        if (f < 0) continue;
        const int a = row_face_a[r * RF + u], side = row_face_side[r * RF + u];
        for (int b = 0; b < fd; ++b) {
            if (face_loc[((int64_t)f * 2 + side) * fd + b] >= 0) continue;
            const int32_t gd = face_dof[(int64_t)f * fd + b];
            const double v = kwf[f] * face_sgn[(int64_t)f * fd + a] * face_sgn[(int64_t)f * fd + b] *
                             face_mass(dim, ref, X, face_v + (int64_t)f * 4, a, b);
            const double2 d = uD[gd];
            if (face_kind[f] == 1) {
                fr += v * d.y;            // -(i v)(d.x + i d.y) = v d.y - i v d.x
                fi -= v * d.x;
                gr += v * d.y;
                gi -= v * d.x;
            } else {                      // -((tre + i tim) v) d
                fr -= v * (tre * d.x - tim * d.y);
                fi -= v * (tre * d.y + tim * d.x);
            }
        }
    }
    f[r] = make_double2(fr, fi);
    fres[r] = make_double2(gr, gi);
}

// ---------------------------------------------------------------------------
// Static condensation of the order-2 cell bubbles (they couple only to the
// edge DOFs of their own cell): per cell D = P_II (4x4), G = P_EI D^{-1}
// (8x4), and the condensed edge matrix S = P_EE - sum_cells G P_IE.
// ---------------------------------------------------------------------------
__global__ void k_condense(int64_t n_cell, const double* __restrict__ ref, const double* __restrict__ X,
                           const int32_t* __restrict__ cells, const int8_t* __restrict__ signs,
                           const double* __restrict__ mu, const double* __restrict__ w2c, double* __restrict__ cinv,
                           double* __restrict__ cg, double* __restrict__ ccor, float* __restrict__ cinv32,
                           float* __restrict__ cg32, int* __restrict__ bad) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_cell) return;
    double hh[3];
    cell_sides(X, 2, cells, c, hh);
    double D[4][8];                              // [D | I] -> [I | D^{-1}]
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            D[i][j] = cell_entry(2, ref, 12, mu[c], w2c[c], hh, 8 + i, 8 + j);
            D[i][4 + j] = i == j ? 1.0 : 0.0;
        }
    for (int k = 0; k < 4; ++k) {
        int p = k;
        for (int i = k + 1; i < 4; ++i)
            if (fabs(D[i][k]) > fabs(D[p][k])) p = i;
        if (!(fabs(D[p][k]) > 0)) { atomicExch(bad, 1); return; }
        if (p != k)
            for (int j = 0; j < 8; ++j) { double t = D[k][j]; D[k][j] = D[p][j]; D[p][j] = t; }
        double inv = 1.0 / D[k][k];
        for (int j = 0; j < 8; ++j) D[k][j] *= inv;
        for (int i = 0; i < 4; ++i)
            if (i != k) {
                double f = D[i][k];
                for (int j = 0; j < 8; ++j) D[i][j] -= f * D[k][j];
            }
    }
    double Di[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = i; j < 4; ++j) {              // symmetrise the inverse of a symmetric block
            double v = 0.5 * (D[i][4 + j] + D[j][4 + i]);
            Di[i][j] = v; Di[j][i] = v;
        }
    double PEI[8][4];
    for (int e = 0; e < 8; ++e)
        for (int k = 0; k < 4; ++k)
            PEI[e][k] = (double)signs[c * 12 + e] * cell_entry(2, ref, 12, mu[c], w2c[c], hh, e, 8 + k);
    double G[8][4];
    for (int e = 0; e < 8; ++e)
        for (int k = 0; k < 4; ++k) {
            double v = 0;
            for (int j = 0; j < 4; ++j) v += PEI[e][j] * Di[j][k];
            G[e][k] = v;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cinv[c * 16 + i * 4 + j] = Di[i][j];
            cinv32[c * 16 + i * 4 + j] = (float)Di[i][j];
        }
    for (int e = 0; e < 8; ++e)
        for (int k = 0; k < 4; ++k) {
            cg[c * 32 + e * 4 + k] = G[e][k];
            cg32[c * 32 + e * 4 + k] = (float)G[e][k];
        }
    for (int e = 0; e < 8; ++e)
        for (int f = e; f < 8; ++f) {              // symmetric correction G P_IE
            double v = 0;
            for (int k = 0; k < 4; ++k) v += G[e][k] * PEI[f][k];
            ccor[c * 64 + e * 8 + f] = v;
            ccor[c * 64 + f * 8 + e] = v;
        }
}

// S values on the SELL pattern: edge row r, edge column: P - sum of cell corrections;
// bubble rows/columns and padding: 0.  Without bubbles S = P.
__global__ void k_condensed_values(int64_t n_loc, int nb, int maxc, int condensed,
                                   const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                                   const uint8_t* __restrict__ pad, const int32_t* __restrict__ row_cell,
                                   const int32_t* __restrict__ row_k, const int32_t* __restrict__ cell_loc,
                                   const uint8_t* __restrict__ is_bub, const double* __restrict__ val,
                                   const double* __restrict__ ccor, double* __restrict__ sval,
                                   float* __restrict__ sval32) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_loc) return;
    int64_t sl = r / SELL_C;
    int lane = (int)(r % SELL_C);
    int64_t base = slice_ptr[sl];
    int w = (int)((slice_ptr[sl + 1] - base) / SELL_C);
    for (int t = 0; t < w; ++t) {
        int64_t idx = base + (int64_t)t * SELL_C + lane;
        double v = 0.0;
        int32_t cc = col[idx];
        if (!pad[idx] && !(condensed && (is_bub[r] || is_bub[cc]))) {
            v = val[idx];
            if (condensed)
                for (int u = 0; u < maxc; ++u) {
                    int32_t c = row_cell[r * maxc + u];
                    if (c < 0) break;
                    int kr = row_k[r * maxc + u];
                    for (int kc = 0; kc < 8; ++kc)
                        if (cell_loc[(int64_t)c * nb + kc] == cc) v -= ccor[(int64_t)c * 64 + kr * 8 + kc];
                }
        }
        sval[idx] = v;
        sval32[idx] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// Twisted level-block-tridiagonal factorisation of S (= P_i, or its edge
// Schur complement for order 2).  With levels l = 0..L-1 (BFS layers of the
// DOF graph, merged up to max_block), S is block tridiagonal with diagonal
// blocks D_l and couplings E_l = S_{l,l-1}, F_l = S_{l,l+1} = E_{l+1}^T.
// Eliminating from both ends towards the middle level k:
//   top    (l = 0..k-1):    S_l = D_l - E_l W_{l-1} E_l^T      (no term for l = 0)
//   bottom (l = L-1..k+1):  S_l = D_l - F_l W_{l+1} F_l^T      (no term for l = L-1)
//   middle:                 S_k = D_k - E_k W_{k-1} E_k^T - F_k W_{k+1} F_k^T
// with W_l = S_l^{-1} by Gauss-Jordan with partial pivoting, all in FP64.
// Each W_l is stored with row stride r4(m_l) (zero padding).
// ---------------------------------------------------------------------------
template <class F>
__device__ bool cta_gauss_jordan(F* W, int m, int ld, int* perm, F* fcol, F* rv, int* ri) {
    __shared__ int s_piv;
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        // pivot: largest |W[i][k]|, i >= k (lowest index on ties)
        F best = -1;
        int bi = -1;
        for (int i = k + threadIdx.x; i < m; i += blockDim.x) {
            F v = W[(int64_t)i * ld + k];
            v = v < 0 ? -v : v;
            if (v > best) { best = v; bi = i; }
        }
        rv[threadIdx.x] = best;
        ri[threadIdx.x] = bi;
        __syncthreads();
        for (int sh = blockDim.x / 2; sh > 0; sh >>= 1) {
            if (threadIdx.x < sh) {
                F o = rv[threadIdx.x + sh];
                int oi = ri[threadIdx.x + sh];
                if (o > rv[threadIdx.x] || (o == rv[threadIdx.x] && oi >= 0 && (ri[threadIdx.x] < 0 || oi < ri[threadIdx.x]))) {
                    rv[threadIdx.x] = o;
                    ri[threadIdx.x] = oi;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_piv = ri[0];
            if (!(rv[0] > 0) || !isfinite((double)rv[0])) s_bad = 1;
            perm[k] = ri[0] < 0 ? k : ri[0];
        }
        __syncthreads();
        if (s_bad) return false;
        int p = s_piv;
        if (p != k)
            for (int j = threadIdx.x; j < m; j += blockDim.x) {
                F a = W[(int64_t)k * ld + j];
                W[(int64_t)k * ld + j] = W[(int64_t)p * ld + j];
                W[(int64_t)p * ld + j] = a;
            }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) fcol[i] = (i == k) ? F(0) : W[(int64_t)i * ld + k];
        __syncthreads();
        F piv = W[(int64_t)k * ld + k];
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            F v = (j == k) ? F(1) : W[(int64_t)k * ld + j];
            W[(int64_t)k * ld + j] = v / piv;
        }
        __syncthreads();
        for (int64_t t = threadIdx.x; t < (int64_t)m * m; t += blockDim.x) {
            int i = (int)(t / m), j = (int)(t % m);
            if (i == k) continue;
            const int64_t o = (int64_t)i * ld + j;
            F a = (j == k) ? F(0) : W[o];
            W[o] = a - fcol[i] * W[(int64_t)k * ld + j];
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int k = m - 1; k >= 0; --k) {
        int p = perm[k];
        if (p != k)
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                F a = W[(int64_t)i * ld + k];
                W[(int64_t)i * ld + k] = W[(int64_t)i * ld + p];
                W[(int64_t)i * ld + p] = a;
            }
        __syncthreads();
    }
    return true;
}

template <class F>
__device__ void extract_block(const Level& L, int64_t c0, int mc, F* dst, int ld, const int64_t* slice_ptr,
                              const int32_t* col, const uint8_t* pad, const double* val) {
    // dst (L.size x mc, row stride ld, padding zeroed) = S rows of level L, columns in [c0, c0 + mc)
    for (int64_t t = threadIdx.x; t < (int64_t)L.size * ld; t += blockDim.x) dst[t] = F(0);
    __syncthreads();
    for (int i = threadIdx.x; i < L.size; i += blockDim.x) {
        int64_t r = L.start + i;
        int64_t sl = r / SELL_C;
        int lane = (int)(r % SELL_C);
        int64_t base = slice_ptr[sl];
        int w = (int)((slice_ptr[sl + 1] - base) / SELL_C);
        for (int t = 0; t < w; ++t) {
            int64_t idx = base + (int64_t)t * SELL_C + lane;
            if (pad[idx]) continue;
            int64_t cc = col[idx];
            if (cc >= c0 && cc < c0 + mc) dst[(int64_t)i * ld + (cc - c0)] = (F)val[idx];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int ld4(int m) { return (m + 3) / 4 * 4; }

// W (m_l rows, stride r4(m_l)) -= C W_n C^T with C = S_{l,n}, the coupling of
// level l to the already-eliminated neighbour n, taken from the level's sparse
// coupling list (side 0: n = l-1, side 1: n = l+1; a few entries per row):
//   T = C W_n  (m_l x m_n, row stride m_n),   W[i][j] -= sum_q T[i][c_q] C[j][c_q].
// T is also the transpose of the neighbour's backward-sweep product
// (H_n = W_n C^T, W_n symmetric), kept at Hn (stride r4(m_n)).
__device__ void schur_update(const Level& L, const Level& N, int side, double* W, const double* Wn, double* tT,
                             const int32_t* __restrict__ cptr, const int32_t* __restrict__ ccol,
                             const double* __restrict__ cval, double* Hn) {
    const int32_t* P = cptr + (side == 0 ? L.eptr : L.fptr);
    const int32_t* Cc = ccol + (side == 0 ? L.eoff : L.foff);
    const double* Cv = cval + (side == 0 ? L.eoff : L.foff);
    const int ml = L.size, mn = N.size, ldn = ld4(mn), ldl = ld4(ml);
    for (int64_t t = threadIdx.x; t < (int64_t)ml * mn; t += blockDim.x) {
        const int i = (int)(t / mn), j = (int)(t % mn);
        double acc = 0;
        for (int p = P[i]; p < P[i + 1]; ++p) acc += Cv[p] * Wn[(int64_t)Cc[p] * ldn + j];
        tT[t] = acc;
        Hn[(int64_t)i * ldn + j] = acc;
    }
    for (int64_t t = threadIdx.x; t < (int64_t)ml * (ldn - mn); t += blockDim.x)   // row padding
        Hn[(t / (ldn - mn)) * ldn + mn + t % (ldn - mn)] = 0;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (int64_t)ml * ml; t += blockDim.x) {
        const int i = (int)(t / ml), j = (int)(t % ml);
        double acc = 0;
        for (int q = P[j]; q < P[j + 1]; ++q) acc += tT[(int64_t)i * mn + Cc[q]] * Cv[q];
        W[(int64_t)i * ldl + j] -= acc;
    }
    __syncthreads();
}

// mid == 0: grid (n_sub, 2), blockIdx.y = 0 the top chain, 1 the bottom chain.
// mid == 1: grid n_sub, the middle level (after both chains).
__global__ void k_bt_factor(int mid, const Sub* __restrict__ subs, const Level* __restrict__ levels,
                            const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                            const uint8_t* __restrict__ pad, const double* __restrict__ sval,
                            const int32_t* __restrict__ cptr, const int32_t* __restrict__ ccol,
                            const double* __restrict__ cval, double* fac, double* tmp_all, int64_t tmp_stride,
                            int* perm_all, int max_m, int* status) {
    extern __shared__ unsigned char smem_raw[];
    double* fcol = reinterpret_cast<double*>(smem_raw);
    double* rv = fcol + max_m;
    int* ri = reinterpret_cast<int*>(rv + blockDim.x);
    const int s = blockIdx.x, chain = mid ? 0 : blockIdx.y;
    const Sub S = subs[s];
    if (S.nlev == 0) return;
    double* tT = tmp_all + ((int64_t)s * 2 + chain) * tmp_stride;
    int* perm = perm_all + ((int64_t)s * 2 + chain) * max_m;
    const int k = S.kmid;
    if (mid) {
        const Level L = levels[S.lev0 + k];
        double* W = fac + L.offW;
        extract_block(L, L.start, L.size, W, ld4(L.size), slice_ptr, col, pad, sval);
        if (k > 0) {
            const Level N = levels[S.lev0 + k - 1];
            schur_update(L, N, 0, W, fac + N.offW, tT, cptr, ccol, cval, fac + N.offH);
        }
        if (k + 1 < S.nlev) {
            const Level N = levels[S.lev0 + k + 1];
            schur_update(L, N, 1, W, fac + N.offW, tT, cptr, ccol, cval, fac + N.offH);
        }
        if (!cta_gauss_jordan(W, L.size, ld4(L.size), perm, fcol, rv, ri) && threadIdx.x == 0) atomicExch(status, 1);
        return;
    }
    const int n = chain == 0 ? k : S.nlev - 1 - k;
    for (int q = 0; q < n; ++q) {
        const int l = chain == 0 ? q : S.nlev - 1 - q;
        const Level L = levels[S.lev0 + l];
        double* W = fac + L.offW;
        extract_block(L, L.start, L.size, W, ld4(L.size), slice_ptr, col, pad, sval);
        if (q > 0) {
            const Level N = levels[S.lev0 + (chain == 0 ? l - 1 : l + 1)];
            schur_update(L, N, chain == 0 ? 0 : 1, W, fac + N.offW, tT, cptr, ccol, cval, fac + N.offH);
        }
        if (!cta_gauss_jordan(W, L.size, ld4(L.size), perm, fcol, rv, ri)) {
            if (threadIdx.x == 0) atomicExch(status, 1);
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// The full 2x2 block operator of Section 3.2 ([[P, -B], [B, P]], the real form
// of T = P + iB) factorised the same way in complex arithmetic: S_l and
// W_l = S_l^{-1} complex (symmetric), couplings real.  2-D only: there B is
// diagonal (the face masses of Gamma^inf and Sigma on the edge rows; the
// order-2 bubbles have no tangential trace), so the level couplings of T are
// those of P and the diagonal blocks gain i B on their diagonal.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__device__ bool cta_gauss_jordan_c(double2* W, int m, int ld, int* perm, double2* fcol, double* rv, int* ri) {
    __shared__ int s_piv;
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        // pivot: largest |W[i][k]|, i >= k (lowest index on ties)
        double best = -1;
        int bi = -1;
        for (int i = k + threadIdx.x; i < m; i += blockDim.x) {
            const double2 v = W[(int64_t)i * ld + k];
            const double a = hypot(v.x, v.y);
            if (a > best) { best = a; bi = i; }
        }
        rv[threadIdx.x] = best;
        ri[threadIdx.x] = bi;
        __syncthreads();
        for (int sh = blockDim.x / 2; sh > 0; sh >>= 1) {
            if (threadIdx.x < sh) {
                const double o = rv[threadIdx.x + sh];
                const int oi = ri[threadIdx.x + sh];
                if (o > rv[threadIdx.x] || (o == rv[threadIdx.x] && oi >= 0 && (ri[threadIdx.x] < 0 || oi < ri[threadIdx.x]))) {
                    rv[threadIdx.x] = o;
                    ri[threadIdx.x] = oi;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_piv = ri[0];
            if (!(rv[0] > 0) || !isfinite(rv[0])) s_bad = 1;
            perm[k] = ri[0] < 0 ? k : ri[0];
        }
        __syncthreads();
        if (s_bad) return false;
        const int p = s_piv;
        if (p != k)
            for (int j = threadIdx.x; j < m; j += blockDim.x) {
                const double2 a = W[(int64_t)k * ld + j];
                W[(int64_t)k * ld + j] = W[(int64_t)p * ld + j];
                W[(int64_t)p * ld + j] = a;
            }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            fcol[i] = (i == k) ? make_double2(0, 0) : W[(int64_t)i * ld + k];
        __syncthreads();
        const double2 piv = W[(int64_t)k * ld + k];
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const double2 v = (j == k) ? make_double2(1, 0) : W[(int64_t)k * ld + j];
            W[(int64_t)k * ld + j] = zdiv(v, piv);
        }
        __syncthreads();
        for (int64_t t = threadIdx.x; t < (int64_t)m * m; t += blockDim.x) {
            const int i = (int)(t / m), j = (int)(t % m);
            if (i == k) continue;
            const int64_t o = (int64_t)i * ld + j;
            const double2 a = (j == k) ? make_double2(0, 0) : W[o];
            const double2 f = zmul(fcol[i], W[(int64_t)k * ld + j]);
            W[o] = make_double2(a.x - f.x, a.y - f.y);
        }
        __syncthreads();
    }
    for (int k = m - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k)
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const double2 a = W[(int64_t)i * ld + k];
                W[(int64_t)i * ld + k] = W[(int64_t)i * ld + p];
                W[(int64_t)i * ld + p] = a;
            }
        __syncthreads();
    }
    return true;
}

// D_l + i B_l of level L (B diagonal: bg + bs of the rows)
__device__ void extract_block_c(const Level& L, double2* dst, int ld, const int64_t* slice_ptr, const int32_t* col,
                                const uint8_t* pad, const double* val, const double* bg, const double* bs) {
    for (int64_t t = threadIdx.x; t < (int64_t)L.size * ld; t += blockDim.x) dst[t] = make_double2(0, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < L.size; i += blockDim.x) {
        const int64_t r = L.start + i;
        const int64_t sl = r / SELL_C;
        const int lane = (int)(r % SELL_C);
        const int64_t base = slice_ptr[sl];
        const int w = (int)((slice_ptr[sl + 1] - base) / SELL_C);
        for (int t = 0; t < w; ++t) {
            const int64_t idx = base + (int64_t)t * SELL_C + lane;
            if (pad[idx]) continue;
            const int64_t cc = col[idx];
            if (cc >= L.start && cc < L.start + L.size) dst[(int64_t)i * ld + (cc - L.start)].x = val[idx];
        }
        dst[(int64_t)i * ld + i].y = bg[r] + bs[r];
    }
    __syncthreads();
}

// W (complex, m_l x r4(m_l)) -= C W_n C^T with the real coupling list C
__device__ void schur_update_c(const Level& L, const Level& N, int side, double2* W, const double2* Wn, double2* tT,
                               const int32_t* __restrict__ cptr, const int32_t* __restrict__ ccol,
                               const double* __restrict__ cval, double2* Hn) {
    const int32_t* P = cptr + (side == 0 ? L.eptr : L.fptr);
    const int32_t* Cc = ccol + (side == 0 ? L.eoff : L.foff);
    const double* Cv = cval + (side == 0 ? L.eoff : L.foff);
    const int ml = L.size, mn = N.size, ldn = ld4(mn), ldl = ld4(ml);
    for (int64_t t = threadIdx.x; t < (int64_t)ml * mn; t += blockDim.x) {
        const int i = (int)(t / mn), j = (int)(t % mn);
        double2 acc = make_double2(0, 0);
        for (int p = P[i]; p < P[i + 1]; ++p) {
            const double2 wv = Wn[(int64_t)Cc[p] * ldn + j];
            acc.x += Cv[p] * wv.x;
            acc.y += Cv[p] * wv.y;
        }
        tT[t] = acc;
        Hn[(int64_t)i * ldn + j] = acc;          // H_n^T, as in schur_update
    }
    for (int64_t t = threadIdx.x; t < (int64_t)ml * (ldn - mn); t += blockDim.x)
        Hn[(t / (ldn - mn)) * ldn + mn + t % (ldn - mn)] = make_double2(0, 0);
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (int64_t)ml * ml; t += blockDim.x) {
        const int i = (int)(t / ml), j = (int)(t % ml);
        double2 acc = make_double2(0, 0);
        for (int q = P[j]; q < P[j + 1]; ++q) {
            const double2 tv = tT[(int64_t)i * mn + Cc[q]];
            acc.x += tv.x * Cv[q];
            acc.y += tv.y * Cv[q];
        }
        W[(int64_t)i * ldl + j].x -= acc.x;
        W[(int64_t)i * ldl + j].y -= acc.y;
    }
    __syncthreads();
}

// As k_bt_factor, in complex arithmetic (mid 0: both chains; mid 1: middle level).
__global__ void k_bt_factor_c(int mid, const Sub* __restrict__ subs, const Level* __restrict__ levels,
                              const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                              const uint8_t* __restrict__ pad, const double* __restrict__ sval,
                              const double* __restrict__ bg, const double* __restrict__ bs,
                              const int32_t* __restrict__ cptr, const int32_t* __restrict__ ccol,
                              const double* __restrict__ cval, double2* fac, double2* tmp_all, int64_t tmp_stride,
                              int* perm_all, int max_m, int* status) {
    extern __shared__ unsigned char smem_raw[];
    double2* fcol = reinterpret_cast<double2*>(smem_raw);
    double* rv = reinterpret_cast<double*>(fcol + max_m);
    int* ri = reinterpret_cast<int*>(rv + blockDim.x);
    const int s = blockIdx.x, chain = mid ? 0 : blockIdx.y;
    const Sub S = subs[s];
    if (S.nlev == 0) return;
    double2* tT = tmp_all + ((int64_t)s * 2 + chain) * tmp_stride;
    int* perm = perm_all + ((int64_t)s * 2 + chain) * max_m;
    const int k = S.kmid;
    if (mid) {
        const Level L = levels[S.lev0 + k];
        double2* W = fac + L.offW;
        extract_block_c(L, W, ld4(L.size), slice_ptr, col, pad, sval, bg, bs);
        if (k > 0) {
            const Level N = levels[S.lev0 + k - 1];
            schur_update_c(L, N, 0, W, fac + N.offW, tT, cptr, ccol, cval, fac + N.offH);
        }
        if (k + 1 < S.nlev) {
            const Level N = levels[S.lev0 + k + 1];
            schur_update_c(L, N, 1, W, fac + N.offW, tT, cptr, ccol, cval, fac + N.offH);
        }
        if (!cta_gauss_jordan_c(W, L.size, ld4(L.size), perm, fcol, rv, ri) && threadIdx.x == 0) atomicExch(status, 1);
        return;
    }
    const int n = chain == 0 ? k : S.nlev - 1 - k;
    for (int q = 0; q < n; ++q) {
        const int l = chain == 0 ? q : S.nlev - 1 - q;
        const Level L = levels[S.lev0 + l];
        double2* W = fac + L.offW;
        extract_block_c(L, W, ld4(L.size), slice_ptr, col, pad, sval, bg, bs);
        if (q > 0) {
            const Level N = levels[S.lev0 + (chain == 0 ? l - 1 : l + 1)];
            schur_update_c(L, N, chain == 0 ? 0 : 1, W, fac + N.offW, tT, cptr, ccol, cval, fac + N.offH);
        }
        if (!cta_gauss_jordan_c(W, L.size, ld4(L.size), perm, fcol, rv, ri)) {
            if (threadIdx.x == 0) atomicExch(status, 1);
            return;
        }
    }
}

__global__ void k_to_float2(int64_t n, const double2* __restrict__ a, float2* __restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void k_gather_slots(int64_t n, const int64_t* __restrict__ slot, const double* __restrict__ v,
                               double* __restrict__ o64, float* __restrict__ o32) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        double x = slot[i] >= 0 ? v[slot[i]] : 0.0;
        o64[i] = x;
        o32[i] = (float)x;
    }
}

// Order-2 gather tables of the condensation steps (see thm_sys::tab_*).  The
// bubbles of a cell are 4 consecutive local rows, the cells of a subdomain
// in bubble-row order; *bad is set if a row breaks that layout.
__global__ void k_cond_tables(int64_t n_loc, int maxc, const uint8_t* __restrict__ is_bub,
                              const int32_t* __restrict__ row_cell, const int32_t* __restrict__ row_k,
                              const int32_t* __restrict__ cell_loc, const int32_t* __restrict__ loc_sub,
                              const Sub* __restrict__ subs, const double* __restrict__ cinv,
                              const double* __restrict__ cg, int32_t* __restrict__ ab, double* __restrict__ av,
                              float* __restrict__ av32, double* __restrict__ cv, float* __restrict__ cv32,
                              int32_t* __restrict__ e8, double* __restrict__ ev, float* __restrict__ ev32,
                              int* __restrict__ bad) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n_loc) return;
    for (int u = 0; u < 2; ++u) ab[u * n_loc + r] = -1;
    for (int u = 0; u < 8; ++u) { av[u * n_loc + r] = 0; av32[u * n_loc + r] = 0; }
    for (int u = 0; u < 4; ++u) { cv[u * n_loc + r] = 0; cv32[u * n_loc + r] = 0; }
    for (int u = 0; u < 8; ++u) { ev[u * n_loc + r] = 0; ev32[u * n_loc + r] = 0; }
    if (!is_bub[r]) {
        int q = 0;
        for (int u = 0; u < maxc; ++u) {
            int32_t c = row_cell[r * maxc + u];
            if (c < 0) break;
            if (u >= 2) { atomicExch(bad, 1); break; }
            const int a = row_k[r * maxc + u];
            const int32_t b0 = cell_loc[(int64_t)c * 12 + 8];
            ab[u * n_loc + r] = b0;
            for (int k = 0; k < 4; ++k, ++q) {
                if (cell_loc[(int64_t)c * 12 + 8 + k] != b0 + k) atomicExch(bad, 1);
                double g = cg[(int64_t)c * 32 + a * 4 + k];
                av[q * n_loc + r] = g;
                av32[q * n_loc + r] = (float)g;
            }
        }
    } else {
        int32_t c = row_cell[r * maxc];
        int k = row_k[r * maxc] - 8;
        const Sub S = subs[loc_sub[r]];
        const int64_t q4 = r - k - (S.off + S.ne);
        if (cell_loc[(int64_t)c * 12 + 8] != r - k || q4 < 0 || (q4 & 3) != 0) atomicExch(bad, 1);
        for (int j = 0; j < 4; ++j) {
            double d = cinv[(int64_t)c * 16 + k * 4 + j];
            cv[j * n_loc + r] = d;
            cv32[j * n_loc + r] = (float)d;
        }
        const int64_t slot = S.cell0 + q4 / 4;
        for (int a = 0; a < 8; ++a) {
            int32_t e = cell_loc[(int64_t)c * 12 + a];
            if (k == 0 && q4 >= 0) e8[slot * 8 + a] = e;
            if (e < 0) continue;
            double g = -cg[(int64_t)c * 32 + a * 4 + k];
            ev[a * n_loc + r] = g;
            ev32[a * n_loc + r] = (float)g;
        }
    }
}

__global__ void k_to_float(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ---------------------------------------------------------------------------
void assemble(thm_sys* s) {
    const thm_mesh* m = s->m;
    cudaStream_t st = s->st;
    const int nb = m->dpc;
    // omega per cell, face and Dirichlet edge (one value unless the mesh holds
    // a batch of independent problems)
    {
        auto prob = [&](int32_t sub) { return (sub < 0 || m->sub_prob.empty()) ? 0 : m->sub_prob[sub]; };
        THM_REQUIRE((int)s->omega_prob.size() == m->n_prob, "one omega per problem required");
        std::vector<double> w2h(m->n_cell), kwh(std::max<int64_t>(1, m->n_face), 0.0);
        std::vector<double> omh(std::max<size_t>(1, m->dir_edges.size()), 0.0);
        std::vector<double> eps;
        if (s->eps.p) s->eps.download(eps, st);
        for (int64_t c = 0; c < m->n_cell; ++c) {
            const double om = s->omega_prob[prob(m->cell_sub[c])];
            w2h[c] = om * om * (eps.empty() ? 1.0 : eps[c]);      // the mass term omega^2 eps_c M_c
        }
        for (int64_t f = 0; f < m->n_face; ++f) {
            const int32_t sb = m->face_sub[2 * f] >= 0 ? m->face_sub[2 * f] : m->face_sub[2 * f + 1];
            kwh[f] = s->kappa * s->omega_prob[prob(sb)];
        }
        if (!m->dir_edges.empty()) {
            const int nv = m->dim == 2 ? 4 : 8;
            std::vector<int32_t> vprob(m->n_vert, 0);
            for (int64_t c = 0; c < m->n_cell; ++c)
                for (int v = 0; v < nv; ++v) vprob[m->cells[c * nv + v]] = prob(m->cell_sub[c]);
            for (size_t t = 0; t < m->dir_edges.size(); ++t)
                omh[t] = s->omega_prob[vprob[m->edge_lo[m->dir_edges[t]]]];
        }
        s->w2c.upload(w2h, st);
        s->kwf.upload(kwh, st);
        s->omd.upload(omh, st);
    }
    s->dev_err.alloc(1);
    s->dev_err.zero(st);
    s->ref.alloc(8 * 144);
    s->ref.zero(st);
    THM_LAUNCH(THM_K_SETUP, st, k_ref_matrices<<<1, 256, 0, st>>>(m->dim, m->order, nb, s->ref.p));
    THM_CUDA(cudaGetLastError());
    s->val64.alloc(m->n_slots);
    s->val32.alloc(m->n_slots);
    const int th = 256;
    auto grid = [&](int64_t n) { return (unsigned)((n + th - 1) / th); };
    THM_LAUNCH(THM_K_SETUP, st, k_assemble<<<grid(m->n_loc), th, 0, st>>>(m->dim, m->n_loc, nb, m->maxc, s->ref.p, m->d_coords.p, m->d_cells.p,
                                              m->d_cell_signs.p, m->d_cell_loc.p, s->mu_inv.p, s->w2c.p,
                                              m->d_slice_ptr.p, m->d_sell_col.p, m->d_sell_pad.p,
                                              m->d_row_cell.p, m->d_row_k.p, s->val64.p, s->val32.p));
    THM_CUDA(cudaGetLastError());
    if (s->trans_re != 0.0) {
        // K_i^loc (no Sigma terms) keeps the values before the real Sigma part is added
        s->valK64.alloc(m->n_slots);
        s->valK32.alloc(m->n_slots);
        THM_CUDA(cudaMemcpyAsync(s->valK64.p, s->val64.p, m->n_slots * sizeof(double), cudaMemcpyDeviceToDevice, st));
        THM_CUDA(cudaMemcpyAsync(s->valK32.p, s->val32.p, m->n_slots * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    s->bg64.alloc(m->n_loc); s->bs64.alloc(m->n_loc);
    s->bg32.alloc(m->n_loc); s->bs32.alloc(m->n_loc);
    const bool sellb = m->dim == 3;
    s->bvg64.alloc(sellb ? m->n_slots : 1); s->bvs64.alloc(sellb ? m->n_slots : 1);
    s->bvg32.alloc(sellb ? m->n_slots : 1); s->bvs32.alloc(sellb ? m->n_slots : 1);
    THM_LAUNCH(THM_K_SETUP, st, k_face_terms<<<grid(m->n_loc), th, 0, st>>>(
        m->dim, m->n_loc, m->fd, s->ref.p, m->d_coords.p, m->d_face_v.p, m->d_face_sgn.p, m->d_face_kind.p,
        m->d_face_loc.p, m->d_row_face.p, m->d_row_face_a.p, m->d_row_face_side.p, m->d_slice_ptr.p,
        m->d_sell_col.p, m->d_sell_pad.p, s->kwf.p, s->trans_re, s->trans_im, s->val64.p, s->val32.p, s->bg64.p,
        s->bs64.p, s->bg32.p, s->bs32.p, s->bvg64.p, s->bvs64.p, s->bvg32.p, s->bvs32.p));
    THM_CUDA(cudaGetLastError());
    const int64_t nterm = (int64_t)m->if_tf.size();
    s->if_val.alloc(nterm > 0 ? nterm : 1);
    if (nterm > 0) {
        THM_LAUNCH(THM_K_SETUP, st, k_iface_vals<<<grid(nterm), th, 0, st>>>(m->dim, nterm, m->fd, s->ref.p, m->d_coords.p,
                                                                            m->d_face_v.p, m->d_face_sgn.p, m->d_if_tf.p,
                                                                            m->d_if_ta.p, m->d_if_tb.p, s->kwf.p,
                                                                            s->if_val.p));
        THM_CUDA(cudaGetLastError());
    }
    s->uD.alloc(m->n_dof);
    s->uD.zero(st);
    if (s->dir_user) {
        const int64_t nd = (int64_t)m->dir_dofs.size();
        if (nd > 0) {
            THM_LAUNCH(THM_K_SETUP, st, k_dirichlet_given<<<grid(nd), th, 0, st>>>(nd, m->d_dir_dofs.p, s->dir_vals.p,
                                                                                  s->uD.p));
            THM_CUDA(cudaGetLastError());
        }
    } else if (!m->dir_edges.empty()) {
        THM_LAUNCH(THM_K_SETUP, st, k_dirichlet<<<grid((int64_t)m->dir_edges.size()), th, 0, st>>>(
            (int64_t)m->dir_edges.size(), m->dim, m->order, m->d_dir_edges.p, m->d_coords.p, m->d_edge_lo.p,
            m->d_edge_hi.p, s->omd.p, s->pol[0], s->pol[1], s->pol[2], s->pol[3], s->pol[4], s->pol[5],
            s->dir[0], s->dir[1], s->dir[2], s->uD.p));
        THM_CUDA(cudaGetLastError());
    }
    // condensed values (order 2) or a copy of P (order 1)
    const int condensed = m->order == 2;
    DArr<double> ccor;
    s->cinv64.alloc(condensed ? m->n_cell * 16 : 1); s->cg64.alloc(condensed ? m->n_cell * 32 : 1);
    s->cinv32.alloc(condensed ? m->n_cell * 16 : 1); s->cg32.alloc(condensed ? m->n_cell * 32 : 1);
    ccor.alloc(condensed ? m->n_cell * 64 : 1);
    if (condensed) {
        DArr<int> bad;
        bad.alloc(1);
        bad.zero(st);
        THM_LAUNCH(THM_K_SETUP, st, k_condense<<<grid(m->n_cell), th, 0, st>>>(m->n_cell, s->ref.p, m->d_coords.p, m->d_cells.p,
                                                     m->d_cell_signs.p, s->mu_inv.p, s->w2c.p, s->cinv64.p, s->cg64.p,
                                                     ccor.p, s->cinv32.p, s->cg32.p, bad.p));
        THM_CUDA(cudaGetLastError());
        std::vector<int> hb;
        bad.download(hb, st);
        if (hb[0]) fail(THM_ESINGULAR, "a cell-bubble block of P_i is singular");
    }
    s->sval64.alloc(m->n_slots);
    s->sval32.alloc(m->n_slots);
    THM_LAUNCH(THM_K_SETUP, st, k_condensed_values<<<grid(m->n_loc), th, 0, st>>>(m->n_loc, nb, m->maxc, condensed, m->d_slice_ptr.p,
                                                      m->d_sell_col.p, m->d_sell_pad.p, m->d_row_cell.p,
                                                      m->d_row_k.p, m->d_cell_loc.p, m->d_loc_is_bub.p,
                                                      s->val64.p, ccor.p, s->sval64.p, s->sval32.p));
    THM_CUDA(cudaGetLastError());
    s->cpl64.alloc(m->cpl_col.size());
    s->cpl32.alloc(m->cpl_col.size());
    THM_LAUNCH(THM_K_SETUP, st, k_gather_slots<<<grid((int64_t)m->cpl_col.size()), th, 0, st>>>((int64_t)m->cpl_col.size(), m->d_cpl_slot.p,
                                                                   s->sval64.p, s->cpl64.p, s->cpl32.p));
    THM_CUDA(cudaGetLastError());
    if (condensed) {
        const size_t n8 = 8 * (size_t)m->n_loc, n4 = 4 * (size_t)m->n_loc;
        s->tab_ab.alloc(2 * (size_t)m->n_loc); s->tab_av64.alloc(n8); s->tab_av32.alloc(n8);
        s->tab_cv64.alloc(n4); s->tab_cv32.alloc(n4);
        s->tab_e8.alloc(8 * (size_t)std::max<int64_t>(1, m->n_bcell)); s->tab_ev64.alloc(n8); s->tab_ev32.alloc(n8);
        DArr<int> bad;
        bad.alloc(1);
        bad.zero(st);
        THM_LAUNCH(THM_K_SETUP, st, k_cond_tables<<<grid(m->n_loc), th, 0, st>>>(m->n_loc, m->maxc, m->d_loc_is_bub.p, m->d_row_cell.p,
                                                     m->d_row_k.p, m->d_cell_loc.p, m->d_loc_sub.p, m->d_subs.p,
                                                     s->cinv64.p, s->cg64.p, s->tab_ab.p, s->tab_av64.p,
                                                     s->tab_av32.p, s->tab_cv64.p, s->tab_cv32.p, s->tab_e8.p,
                                                     s->tab_ev64.p, s->tab_ev32.p, bad.p));
        THM_CUDA(cudaGetLastError());
        std::vector<int> hb;
        bad.download(hb, st);
        THM_REQUIRE(hb[0] == 0, "internal: order-2 bubble rows not in cell groups of 4");
    }
    s->f_loc.alloc(m->n_loc);
    s->f_res.alloc(m->n_loc);
    THM_LAUNCH(THM_K_SETUP, st, k_lifting<<<grid(m->n_loc), th, 0, st>>>(
        m->dim, m->n_loc, nb, m->maxc, s->ref.p, m->d_coords.p, m->d_cells.p, m->d_cell_signs.p, m->d_cell_loc.p,
        m->d_cell_dofs.p, s->mu_inv.p, s->w2c.p, m->d_row_cell.p, m->d_row_k.p, s->uD.p, m->fd, m->d_face_v.p,
        m->d_face_dof.p, m->d_face_sgn.p, m->d_face_loc.p, m->d_row_face.p, m->d_row_face_a.p, m->d_row_face_side.p,
        m->d_face_kind.p, s->kwf.p, s->trans_re, s->trans_im, s->f_loc.p, s->f_res.p));
    THM_CUDA(cudaGetLastError());
    THM_CUDA(cudaStreamSynchronize(st));
}

static void factor64(thm_sys* s) {
    const thm_mesh* m = s->m;
    cudaStream_t st = s->st;
    s->fac64.alloc(m->fac_elems);
    s->fac64.zero(st);
    DArr<double> tmp;
    const int64_t stride = (int64_t)m->max_m * m->max_m;      // T = C W_n of one chain
    tmp.alloc((size_t)stride * m->n_sub * 2);
    DArr<int> perm, status;
    perm.alloc((size_t)m->max_m * m->n_sub * 2);
    status.alloc(1);
    status.zero(st);
    const int threads = 512;
    size_t smem = (size_t)m->max_m * sizeof(double) + threads * (sizeof(double) + sizeof(int));
    if (smem > 48 * 1024)
        THM_CUDA(cudaFuncSetAttribute(k_bt_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    THM_LAUNCH(THM_K_SETUP, st, k_bt_factor<<<dim3(m->n_sub, 2), threads, smem, st>>>(
        0, m->d_subs.p, m->d_levels.p, m->d_slice_ptr.p, m->d_sell_col.p, m->d_sell_pad.p, s->sval64.p, m->d_cpl_ptr.p,
        m->d_cpl_col.p, s->cpl64.p, s->fac64.p, tmp.p, stride, perm.p, m->max_m, status.p));
    THM_LAUNCH(THM_K_SETUP, st, k_bt_factor<<<m->n_sub, threads, smem, st>>>(
        1, m->d_subs.p, m->d_levels.p, m->d_slice_ptr.p, m->d_sell_col.p, m->d_sell_pad.p, s->sval64.p, m->d_cpl_ptr.p,
        m->d_cpl_col.p, s->cpl64.p, s->fac64.p, tmp.p, stride, perm.p, m->max_m, status.p));
    THM_CUDA(cudaGetLastError());
    std::vector<int> hs;
    status.download(hs, st);
    if (hs[0] != 0)
        fail(THM_ESINGULAR, "a diagonal block of P_i = A_i - omega^2 M_i is singular "
                            "(omega^2 is a natural-boundary eigenvalue of a subdomain block)");
}

static void factor_full64(thm_sys* s) {
    const thm_mesh* m = s->m;
    cudaStream_t st = s->st;
    THM_REQUIRE(m->dim == 2, "the full 2x2 block preconditioner is built for 2-D meshes (diagonal B) only");
    s->facc64.alloc(m->fac_elems);
    s->facc64.zero(st);
    DArr<double2> tmp;
    const int64_t stride = (int64_t)m->max_m * m->max_m;
    tmp.alloc((size_t)stride * m->n_sub * 2);
    DArr<int> perm, status;
    perm.alloc((size_t)m->max_m * m->n_sub * 2);
    status.alloc(1);
    status.zero(st);
    const int threads = 512;
    size_t smem = (size_t)m->max_m * sizeof(double2) + threads * (sizeof(double) + sizeof(int));
    if (smem > 48 * 1024)
        THM_CUDA(cudaFuncSetAttribute(k_bt_factor_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    THM_LAUNCH(THM_K_SETUP, st, k_bt_factor_c<<<dim3(m->n_sub, 2), threads, smem, st>>>(
        0, m->d_subs.p, m->d_levels.p, m->d_slice_ptr.p, m->d_sell_col.p, m->d_sell_pad.p, s->sval64.p, s->bg64.p,
        s->bs64.p, m->d_cpl_ptr.p, m->d_cpl_col.p, s->cpl64.p, s->facc64.p, tmp.p, stride, perm.p, m->max_m, status.p));
    THM_LAUNCH(THM_K_SETUP, st, k_bt_factor_c<<<m->n_sub, threads, smem, st>>>(
        1, m->d_subs.p, m->d_levels.p, m->d_slice_ptr.p, m->d_sell_col.p, m->d_sell_pad.p, s->sval64.p, s->bg64.p,
        s->bs64.p, m->d_cpl_ptr.p, m->d_cpl_col.p, s->cpl64.p, s->facc64.p, tmp.p, stride, perm.p, m->max_m, status.p));
    THM_CUDA(cudaGetLastError());
    std::vector<int> hs;
    status.download(hs, st);
    if (hs[0] != 0) fail(THM_ESINGULAR, "a diagonal block of the complex subdomain operator T_i is singular");
}

// The full-block factors (complex), FP64 and for the mixed mode FP32.
void ensure_factor_full(thm_sys* s, bool fp32) {
    if (!s->facc64_ok) { factor_full64(s); s->facc64_ok = true; }
    if (fp32 && !s->facc32_ok) {
        s->facc32.alloc(s->facc64.n);
        THM_LAUNCH(THM_K_SETUP, 0, k_to_float2<<<(unsigned)((s->facc64.n + 255) / 256), 256, 0, s->st>>>(
            (int64_t)s->facc64.n, s->facc64.p, s->facc32.p));
        THM_CUDA(cudaGetLastError());
        s->facc32_ok = true;
    }
}

// The factorisation runs in FP64 for both modes (pivots and Schur updates in
// FP64); the mixed mode stores the inverse blocks rounded to FP32.
void ensure_factor(thm_sys* s, bool fp32) {
    if (!s->fac64_ok) { factor64(s); s->fac64_ok = true; }
    if (fp32 && !s->fac32_ok) {
        s->fac32.alloc(s->fac64.n);
        THM_LAUNCH(THM_K_SETUP, 0, k_to_float<<<(unsigned)((s->fac64.n + 255) / 256), 256, 0, s->st>>>((int64_t)s->fac64.n, s->fac64.p, s->fac32.p));
        THM_CUDA(cudaGetLastError());
        s->fac32_ok = true;
    }
}

}  // namespace thm

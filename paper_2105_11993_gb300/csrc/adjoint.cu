// Discrete adjoint of the DDM solve (no counterpart in the paper).
//
// For a real loss L(u) with a = dL/du (Wirtinger) and K_FF u_F = -K_FD u_D:
//   K_FF lambda = a_F            (K is complex symmetric: the forward DDM solve)
//   dL/dmu_c  = -2 Re(lambda_c^T A_c u_c)
//   dL/domega = -2 Re(lambda^T [(-2 omega M + i kappa M_Gamma) u + K du_D/domega])
//               + 2 Re(a . du_D/domega)
//   dL/dkappa = -2 Re(lambda^T (i omega M_Gamma) u)
// with lambda = 0 on Dirichlet DOFs.  The forward solution u is an input (it is
// recomputed by the caller, not stored with Krylov bases).
#include <chrono>
#include <cmath>

#include "element.cuh"
#include "solver.cuh"

namespace thm {

__constant__ double c_ag_x[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                                 -0.1834346424956498, 0.1834346424956498,  0.5255324099163290,
                                 0.7966664774136267,  0.9602898564975363};
__constant__ double c_ag_w[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                                 0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                                 0.2223810344533745, 0.1012285362903763};

__global__ void k_adj_rhs(int64_t n_loc, const int64_t* __restrict__ gdof, const uint8_t* __restrict__ owner,
                          const double2* __restrict__ a, double2* __restrict__ src) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n_loc) src[r] = owner[r] ? a[gdof[r]] : make_double2(0, 0);
}

// d u_D / d omega: the tangential moments of d/dw [pol exp(-i w dir.x)].
__global__ void k_dirichlet_dw(int64_t n_de, int dim, int order, const int64_t* __restrict__ edges,
                               const double* __restrict__ X, const int64_t* __restrict__ elo,
                               const int64_t* __restrict__ ehi, double omega, double pr0, double pi0, double pr1,
                               double pi1, double pr2, double pi2, double d0, double d1, double d2,
                               double2* __restrict__ duD) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_de) return;
    int64_t e = edges[t];
    double xl[3] = {0, 0, 0}, tv[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
        xl[k] = X[elo[e] * dim + k];
        tv[k] = X[ehi[e] * dim + k] - xl[k];
    }
    double l = sqrt(tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2]);
    double ptr = (pr0 * tv[0] + pr1 * tv[1] + pr2 * tv[2]) / l;
    double pti = (pi0 * tv[0] + pi1 * tv[1] + pi2 * tv[2]) / l;
    double m0r = 0, m0i = 0, m1r = 0, m1i = 0;
    for (int q = 0; q < 8; ++q) {
        double s = 0.5 * (c_ag_x[q] + 1.0), wq = 0.5 * c_ag_w[q];
        double dx = d0 * (xl[0] + s * tv[0]) + d1 * (xl[1] + s * tv[1]) + d2 * (xl[2] + s * tv[2]);
        double sn, cs;
        sincos(-omega * dx, &sn, &cs);
        double er = ptr * cs - pti * sn, ei = ptr * sn + pti * cs;     // E_t
        double dr = dx * ei, di = -dx * er;                             // -i dx E_t
        m0r += wq * dr; m0i += wq * di;
        m1r += wq * dr * (1.0 - 2.0 * s); m1i += wq * di * (1.0 - 2.0 * s);
    }
    if (order == 1) {
        duD[e] = make_double2(l * m0r, l * m0i);
    } else {
        duD[2 * e] = make_double2(l * m0r, l * m0i);
        duD[2 * e + 1] = make_double2(3.0 * l * m1r, 3.0 * l * m1i);
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Per cell: dL/dmu_c and the cell's share of dL/domega (volume terms;
// K_c = mu_c A_c - omega^2 eps_c M_c).
__global__ void k_adj_cells(int dim, int64_t n_cell, int nb, const double* __restrict__ ref,
                            const double* __restrict__ X, const int32_t* __restrict__ cells,
                            const int32_t* __restrict__ cdofs, const int8_t* __restrict__ signs,
                            const double* __restrict__ mu, const double* __restrict__ w2c, double omega,
                            const double2* __restrict__ lam,
                            const double2* __restrict__ u, const double2* __restrict__ duD,
                            double* __restrict__ gmu, double* __restrict__ gw) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_cell) return;
    double h[3];
    cell_sides(X, dim, cells, c, h);
    double2 lc[12], uc[12], dc[12];
    for (int i = 0; i < nb; ++i) {
        double s = (double)signs[c * nb + i];
        int32_t d = cdofs[c * nb + i];
        lc[i] = make_double2(s * lam[d].x, s * lam[d].y);
        uc[i] = make_double2(s * u[d].x, s * u[d].y);
        dc[i] = make_double2(s * duD[d].x, s * duD[d].y);
    }
    double2 sA = make_double2(0, 0), sM = make_double2(0, 0), sD = make_double2(0, 0);
    const double w2 = w2c[c];                   // omega^2 eps_c: the cell's mass-term weight
    for (int i = 0; i < nb; ++i) {
        double2 tA = make_double2(0, 0), tM = make_double2(0, 0), tD = make_double2(0, 0);
        for (int j = 0; j < nb; ++j) {
            double A, M;
            cell_am(dim, ref, nb, h, i, j, A, M);
            tA.x += A * uc[j].x; tA.y += A * uc[j].y;
            tM.x += M * uc[j].x; tM.y += M * uc[j].y;
            double K = mu[c] * A - w2 * M;
            tD.x += K * dc[j].x; tD.y += K * dc[j].y;
        }
        double2 p = cmul(lc[i], tA), q = cmul(lc[i], tM), r = cmul(lc[i], tD);
        sA.x += p.x; sA.y += p.y;
        sM.x += q.x; sM.y += q.y;
        sD.x += r.x; sD.y += r.y;
    }
    gmu[c] = -2.0 * sA.x;
    gw[c] = -2.0 * (-2.0 * (w2 / omega) * sM.x) - 2.0 * sD.x;      // dK_c/domega = -2 omega eps_c M_c
}

// Gamma^inf face share of dL/domega and of dL/dkappa: with m_f the signed face
// mass and K's face term i kappa omega m_f,
//   dL/domega: -2 Re(lambda^T (i kappa m_f) u) - 2 Re(lambda^T (i kappa omega m_f) du_D/domega)
//   dL/dkappa: -2 Re(lambda^T (i omega m_f) u)   (the Dirichlet data do not depend on kappa)
// (u includes the Dirichlet values; in 3-D an impedance face may hold edges
// of the Dirichlet boundary, so both terms reach Dirichlet columns).
__global__ void k_adj_faces(int dim, int64_t n_face, int fd, const double* __restrict__ ref,
                            const double* __restrict__ X, const int32_t* __restrict__ face_v,
                            const int32_t* __restrict__ face_dof, const int8_t* __restrict__ face_sgn,
                            const int8_t* __restrict__ face_kind, double kappa, double omega,
                            const double2* __restrict__ lam, const double2* __restrict__ u,
                            const double2* __restrict__ duD, double* __restrict__ gw, double* __restrict__ gk) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= n_face) return;
    if (face_kind[f] != 1) { gw[f] = 0; gk[f] = 0; return; }
    double2 s1 = make_double2(0, 0), s2 = make_double2(0, 0);
    for (int a = 0; a < fd; ++a) {
        const int32_t da = face_dof[f * fd + a];
        const double2 la = lam[da];
        for (int b = 0; b < fd; ++b) {
            const int32_t db = face_dof[f * fd + b];
            const double mab = face_sgn[f * fd + a] * face_sgn[f * fd + b] *
                               face_mass(dim, ref, X, face_v + f * 4, a, b);
            const double2 p = cmul(la, u[db]), q = cmul(la, duD[db]);
            s1.x += mab * p.x; s1.y += mab * p.y;
            s2.x += mab * q.x; s2.y += mab * q.y;
        }
    }
    gw[f] = 2.0 * kappa * s1.y + 2.0 * kappa * omega * s2.y;      // -2 Re(i c z) = 2 c Im(z)
    gk[f] = 2.0 * omega * s1.y;                                    // dK/dkappa = i omega M_Gamma
}

__global__ void k_adj_dir(int64_t n_dof, const double2* __restrict__ a, const double2* __restrict__ duD,
                          double* __restrict__ gw) {
    int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (d < n_dof) gw[d] = 2.0 * (a[d].x * duD[d].x - a[d].y * duD[d].y);
}

__global__ void k_sum_blocks(int64_t n, const double* __restrict__ x, double* __restrict__ part) {
    __shared__ double sw[32];
    double s = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) s += x[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sw[q];
        part[blockIdx.x] = t;
    }
}

static double device_sum(cudaStream_t st, const double* x, int64_t n, DArr<double>& part) {
    const int nbk = 256;
    THM_LAUNCH(THM_K_DDM, st, k_sum_blocks<<<nbk, 256, 0, st>>>(n, x, part.p));
    std::vector<double> h(nbk);
    THM_CUDA(cudaMemcpyAsync(h.data(), part.p, nbk * sizeof(double), cudaMemcpyDeviceToHost, st));
    THM_CUDA(cudaStreamSynchronize(st));
    double t = 0;
    for (double v : h) t += v;
    return t;
}

int adjoint(thm_sys* s, const thm_solve_opts* opts, const double2* u, const double2* a, double* grad_mu,
            double* grad_omega, double* grad_kappa, thm_stats* stats) {
    auto t0 = std::chrono::steady_clock::now();
    const thm_mesh* m = s->m;
    THM_REQUIRE(m->n_prob == 1, "the adjoint takes a single problem, not a batch");
    cudaStream_t st = s->st;
    SolveCfg c = make_cfg(opts);
    prepare(s, c);
    auto nb = [](int64_t n) { return (unsigned)((n + 255) / 256); };
    DArr<double2> rhs, lam, duD;
    DArr<double> gw_cell, gw_face, gk_face, gw_dof, part;
    rhs.alloc(m->n_loc); lam.alloc(m->n_dof); duD.alloc(m->n_dof);
    gw_cell.alloc(m->n_cell); gw_face.alloc(std::max<int64_t>(1, m->n_face)); gw_dof.alloc(m->n_dof);
    gk_face.alloc(std::max<int64_t>(1, m->n_face));
    part.alloc(256);
    gw_face.zero(st);
    gk_face.zero(st);
    THM_LAUNCH(THM_K_DDM, st, k_adj_rhs<<<nb(m->n_loc), 256, 0, st>>>(m->n_loc, m->d_loc_gdof.p, m->d_loc_is_owner.p, a, rhs.p));
    RunStats rs;
    double rel = 0;
    int rc = solve_rhs(s, c, rhs.p, rhs.p, nullptr, lam.p, rs, rel);
    duD.zero(st);
    // caller-given Dirichlet values (thm_assemble_dirichlet) do not depend on omega
    if (!m->dir_edges.empty() && !s->dir_user)
        THM_LAUNCH(THM_K_DDM, st, k_dirichlet_dw<<<nb((int64_t)m->dir_edges.size()), 256, 0, st>>>(
            (int64_t)m->dir_edges.size(), m->dim, m->order, m->d_dir_edges.p, m->d_coords.p, m->d_edge_lo.p,
            m->d_edge_hi.p, s->omega, s->pol[0], s->pol[1], s->pol[2], s->pol[3], s->pol[4], s->pol[5], s->dir[0],
            s->dir[1], s->dir[2], duD.p));
    THM_LAUNCH(THM_K_DDM, st, k_adj_cells<<<nb(m->n_cell), 256, 0, st>>>(m->dim, m->n_cell, m->dpc, s->ref.p, m->d_coords.p,
                                                                        m->d_cells.p, m->d_cell_dofs.p, m->d_cell_signs.p,
                                                                        s->mu_inv.p, s->w2c.p, s->omega, lam.p, u, duD.p, grad_mu,
                                                                        gw_cell.p));
    if (m->n_face > 0)
        THM_LAUNCH(THM_K_DDM, st, k_adj_faces<<<nb(m->n_face), 256, 0, st>>>(
            m->dim, m->n_face, m->fd, s->ref.p, m->d_coords.p, m->d_face_v.p, m->d_face_dof.p, m->d_face_sgn.p,
            m->d_face_kind.p, s->kappa, s->omega, lam.p, u, duD.p, gw_face.p, gk_face.p));
    THM_LAUNCH(THM_K_DDM, st, k_adj_dir<<<nb(m->n_dof), 256, 0, st>>>(m->n_dof, a, duD.p, gw_dof.p));
    THM_CUDA(cudaGetLastError());
    *grad_omega = device_sum(st, gw_cell.p, m->n_cell, part) + device_sum(st, gw_face.p, std::max<int64_t>(1, m->n_face), part) +
                  device_sum(st, gw_dof.p, m->n_dof, part);
    if (grad_kappa) *grad_kappa = device_sum(st, gk_face.p, std::max<int64_t>(1, m->n_face), part);
    double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    fill_stats(rs, rel, sec, stats);
    return rc;
}

}  // namespace thm

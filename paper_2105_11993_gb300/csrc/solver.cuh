// Host-side interface between the solve driver and the adjoint.
#pragma once

#include "common.cuh"

namespace thm {

struct SolveCfg {
    bool fp32;
    double inner_tol, outer_tol, rtol;
    double cycle_tol;          // mixed: relative tolerance of one FP32 GMRES cycle
    int m_in, m_out, inner_maxit, outer_maxit, max_refine;
    int relax;
    int outer_method;          // THM_OUTER_GMRES / THM_OUTER_JACOBI
    int precond;               // THM_PRECOND_BLOCKDIAG / THM_PRECOND_FULL
};

struct RunStats {
    int outer = 0, sweeps = 0, refine = 0, max_inner = 0;
    int64_t inner = 0, dof_iters = 0;
    int status = THM_OK;
};

SolveCfg make_cfg(const thm_solve_opts* o);
void prepare(thm_sys* s, const SolveCfg& c);
int solve_rhs(thm_sys* s, const SolveCfg& c, const double2* f_src, const double2* f_loc, const double2* u0,
              double2* u, RunStats& rs, double& rel);
void fill_stats(const RunStats& rs, double rel, double sec, thm_stats* stats);

}  // namespace thm

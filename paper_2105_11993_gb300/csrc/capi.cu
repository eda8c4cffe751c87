// extern "C" entry points: argument checks, error codes, thread-local messages.
#include <cmath>
#include <atomic>
#include <new>

#include "common.cuh"

namespace thm {
int solve(thm_sys* s, const thm_solve_opts* opts, double2* u, thm_stats* stats);
void apply_local(thm_sys* s, int op, int mode, const double2* x, double2* y);
int sweep_diag(thm_sys* s, const thm_solve_opts* opts, int with_sources, const double2* g_in, double2* g_out,
               double2* uloc, thm_stats* stats);
int adjoint(thm_sys* s, const thm_solve_opts* opts, const double2* u, const double2* rhs, double* grad_mu,
            double* grad_omega, double* grad_kappa, thm_stats* stats);

extern std::atomic<long long> g_launches;
static thread_local std::string g_msg;

void fail(int code, const std::string& msg) { throw Error{code, msg}; }
void set_last_error(const std::string& msg) { g_msg = msg; }

template <class Fn>
static int guarded(Fn&& fn) {
    try {
        g_msg.clear();
        return fn();
    } catch (const Error& e) {
        g_msg = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        g_msg = "host allocation failed";
        return THM_ENOMEM;
    } catch (const std::exception& e) {
        g_msg = e.what();
        return THM_EINVAL;
    }
}

static void require_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0)
        fail(THM_ECUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
}

}  // namespace thm

using namespace thm;

extern "C" {

const char* thm_last_error(void) { return g_msg.c_str(); }

int thm_mesh_create(thm_mesh** out, int dim, int order, int64_t n_vert, const double* coords, int64_t n_cell,
                    const int64_t* cells, const int32_t* cell_sub, int64_t n_bface, const int64_t* bfaces,
                    const uint8_t* btag, int max_block) {
    return guarded([&]() -> int {
        THM_REQUIRE(out, "out is NULL");
        *out = nullptr;
        THM_REQUIRE(dim == 2 || dim == 3, "dim must be 2 or 3");
        THM_REQUIRE(order == 1 || (order == 2 && dim == 2), "order must be 1 (2-D/3-D) or 2 (2-D)");
        THM_REQUIRE(n_vert > 0 && n_cell > 0 && n_bface >= 0, "empty mesh");
        THM_REQUIRE(coords && cells && cell_sub && (n_bface == 0 || (bfaces && btag)), "NULL array");
        THM_REQUIRE(n_vert < (int64_t)INT32_MAX && n_cell < (int64_t)INT32_MAX / 16, "mesh too large");
        require_device();
        const int nv = dim == 2 ? 4 : 8;
        for (int64_t i = 0; i < n_cell * nv; ++i)
            THM_REQUIRE(cells[i] >= 0 && cells[i] < n_vert, "cell vertex id out of range");
        int32_t smax = -1;
        for (int64_t c = 0; c < n_cell; ++c) {
            THM_REQUIRE(cell_sub[c] >= 0, "negative subdomain id");
            smax = std::max(smax, cell_sub[c]);
        }
        for (int64_t i = 0; i < n_vert * dim; ++i) THM_REQUIRE(std::isfinite(coords[i]), "non-finite coordinate");
        thm_mesh* m = new thm_mesh();
        try {
            m->dim = dim;
            m->order = order;
            m->max_block = max_block > 0 ? max_block : (order == 1 ? 1024 : 160);
            m->n_vert = n_vert;
            m->n_cell = n_cell;
            m->n_bface = n_bface;
            m->n_sub = smax + 1;
            m->coords.assign(coords, coords + n_vert * dim);
            m->cells.assign(cells, cells + n_cell * nv);
            m->cell_sub.assign(cell_sub, cell_sub + n_cell);
            const int fv = dim == 2 ? 2 : 4;
            m->bfaces.assign(bfaces, bfaces + n_bface * fv);
            m->btag.assign(btag, btag + n_bface);
            build_mesh(m);
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
        return THM_OK;
    });
}

int thm_mesh_info(const thm_mesh* m, int64_t* n_dof, int64_t* n_edge, int32_t* n_sub, int32_t* dofs_per_cell,
                  int64_t* dof_of_cell, int8_t* sign_of_cell) {
    return guarded([&]() -> int {
        THM_REQUIRE(m, "mesh is NULL");
        if (n_dof) *n_dof = m->n_dof;
        if (n_edge) *n_edge = m->n_edge;
        if (n_sub) *n_sub = m->n_sub;
        if (dofs_per_cell) *dofs_per_cell = m->dpc;
        if (dof_of_cell) std::copy(m->cell_dofs.begin(), m->cell_dofs.end(), dof_of_cell);
        if (sign_of_cell) std::copy(m->cell_signs.begin(), m->cell_signs.end(), sign_of_cell);
        return THM_OK;
    });
}

void thm_mesh_destroy(thm_mesh* m) { delete m; }

static int assemble_common(thm_sys** out, const thm_mesh* m, const double* mu_inv, int mu_inv_on_device,
                           const std::vector<double>& omegas, double kappa, const double* pol, const double* dir,
                           void* stream, const thm_assemble_opts* ao = nullptr) {
    return guarded([&]() -> int {
        THM_REQUIRE(out && m && mu_inv, "NULL argument");
        const double* u_dir = ao ? ao->u_dir : nullptr;
        const int u_dir_on_device = ao ? ao->u_dir_on_device : 0;
        const bool given = u_dir != nullptr;
        THM_REQUIRE(!given || m->n_prob == 1, "caller-given Dirichlet values: single problems only");
        THM_REQUIRE(given || (pol && dir), "NULL argument (plane-wave polarisation / direction)");
        *out = nullptr;
        THM_REQUIRE((int)omegas.size() == m->n_prob, "one omega per problem required");
        for (double w : omegas) THM_REQUIRE(std::isfinite(w) && w > 0, "omega must be > 0");
        THM_REQUIRE(std::isfinite(kappa) && kappa >= 0, "kappa must be >= 0");
        thm_sys* s = new thm_sys();
        try {
            s->m = m;
            s->st = (cudaStream_t)stream;
            s->omega = omegas[0];
            s->omega_prob = omegas;
            s->kappa = kappa;
            if (given) {
                const int64_t nd = (int64_t)m->dir_dofs.size();
                s->dir_user = true;
                s->dir_vals.alloc(nd > 0 ? nd : 1);
                if (nd > 0) {
                    if (u_dir_on_device) {
                        THM_CUDA(cudaMemcpyAsync(s->dir_vals.p, u_dir, nd * sizeof(double2), cudaMemcpyDeviceToDevice,
                                                 s->st));
                    } else {
                        for (int64_t i = 0; i < 2 * nd; ++i)
                            THM_REQUIRE(std::isfinite(u_dir[i]), "non-finite Dirichlet value");
                        THM_CUDA(cudaMemcpyAsync(s->dir_vals.p, u_dir, nd * sizeof(double2), cudaMemcpyHostToDevice,
                                                 s->st));
                    }
                }
            } else {
                for (int k = 0; k < m->dim; ++k) {
                    s->pol[2 * k] = pol[2 * k];
                    s->pol[2 * k + 1] = pol[2 * k + 1];
                    s->dir[k] = dir[k];
                }
            }
            if (ao && (ao->trans_re != 0.0 || ao->trans_im != 0.0)) {
                THM_REQUIRE(std::isfinite(ao->trans_re) && std::isfinite(ao->trans_im),
                            "non-finite transmission coefficient");
                s->trans_re = ao->trans_re;
                s->trans_im = ao->trans_im;
            }
            if (ao && ao->eps) {
                s->eps.alloc(m->n_cell);
                std::vector<double> e(m->n_cell);
                if (ao->eps_on_device)
                    THM_CUDA(cudaMemcpyAsync(e.data(), ao->eps, m->n_cell * sizeof(double), cudaMemcpyDeviceToHost,
                                             s->st));
                else
                    std::copy(ao->eps, ao->eps + m->n_cell, e.begin());
                THM_CUDA(cudaStreamSynchronize(s->st));
                for (double v : e) THM_REQUIRE(std::isfinite(v) && v > 0, "eps must be finite and > 0");
                THM_CUDA(cudaMemcpyAsync(s->eps.p, e.data(), m->n_cell * sizeof(double), cudaMemcpyHostToDevice, s->st));
                THM_CUDA(cudaStreamSynchronize(s->st));
            }
            s->mu_inv.alloc(m->n_cell);
            if (mu_inv_on_device) {
                THM_CUDA(cudaMemcpyAsync(s->mu_inv.p, mu_inv, m->n_cell * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
            } else {
                for (int64_t c = 0; c < m->n_cell; ++c)
                    THM_REQUIRE(std::isfinite(mu_inv[c]) && mu_inv[c] > 0, "mu_inv must be finite and > 0");
                THM_CUDA(cudaMemcpyAsync(s->mu_inv.p, mu_inv, m->n_cell * sizeof(double), cudaMemcpyHostToDevice, s->st));
            }
            m->assembled = true;
            assemble(s);
        } catch (...) {
            delete s;
            throw;
        }
        *out = s;
        return THM_OK;
    });
}

int thm_assemble(thm_sys** out, const thm_mesh* m, const double* mu_inv, int mu_inv_on_device, double omega,
                 double kappa, const double* pol, const double* dir, void* stream) {
    if (m && m->n_prob != 1) {
        set_last_error("the mesh holds a batch of problems: use thm_assemble_batch");
        if (out) *out = nullptr;
        return THM_EINVAL;
    }
    return assemble_common(out, m, mu_inv, mu_inv_on_device, std::vector<double>{omega}, kappa, pol, dir, stream);
}

int thm_assemble_dirichlet(thm_sys** out, const thm_mesh* m, const double* mu_inv, int mu_inv_on_device,
                           double omega, double kappa, const double* u_dir, int u_dir_on_device, void* stream) {
    if (m && m->n_prob != 1) {
        set_last_error("thm_assemble_dirichlet takes a single problem, not a batch");
        if (out) *out = nullptr;
        return THM_EINVAL;
    }
    if (m && !m->dir_dofs.empty() && !u_dir) {
        set_last_error("u_dir is NULL but the mesh has Dirichlet DOFs");
        if (out) *out = nullptr;
        return THM_EINVAL;
    }
    static const double none = 0.0;
    thm_assemble_opts ao{};
    ao.u_dir = u_dir ? u_dir : &none;
    ao.u_dir_on_device = u_dir_on_device;
    return assemble_common(out, m, mu_inv, mu_inv_on_device, std::vector<double>{omega}, kappa, nullptr, nullptr,
                           stream, &ao);
}

int thm_assemble_ex(thm_sys** out, const thm_mesh* m, const double* mu_inv, int mu_inv_on_device,
                    const double* omega, double kappa, const double* pol, const double* dir,
                    const thm_assemble_opts* opts, void* stream) {
    if (!m || !omega) {
        set_last_error("NULL argument");
        if (out) *out = nullptr;
        return THM_EINVAL;
    }
    thm_assemble_opts ao{};
    if (opts) ao = *opts;
    return assemble_common(out, m, mu_inv, mu_inv_on_device, std::vector<double>(omega, omega + m->n_prob), kappa,
                           pol, dir, stream, &ao);
}

int thm_mesh_dirichlet_dofs(const thm_mesh* m, int64_t* n_dir, int64_t* ids) {
    return guarded([&]() -> int {
        THM_REQUIRE(m, "mesh is NULL");
        if (n_dir) *n_dir = (int64_t)m->dir_dofs.size();
        if (ids) std::copy(m->dir_dofs.begin(), m->dir_dofs.end(), ids);
        return THM_OK;
    });
}

int thm_mesh_set_problems(thm_mesh* m, int32_t n_prob, const int32_t* sub_problem) {
    return guarded([&]() -> int {
        THM_REQUIRE(m && sub_problem, "NULL argument");
        THM_REQUIRE(!m->assembled, "thm_mesh_set_problems must come before the first thm_assemble on this mesh");
        THM_REQUIRE(n_prob >= 1 && n_prob <= m->n_sub, "n_prob must be in [1, n_sub]");
        std::vector<int32_t> sp(sub_problem, sub_problem + m->n_sub);
        std::vector<int64_t> nsub_of(n_prob, 0);
        for (int i = 0; i < m->n_sub; ++i) {
            THM_REQUIRE(sp[i] >= 0 && sp[i] < n_prob, "problem id out of range");
            THM_REQUIRE(i == 0 || sp[i] >= sp[i - 1], "problems must own contiguous, increasing ranges of subdomain ids");
            nsub_of[sp[i]]++;
        }
        for (int p = 0; p < n_prob; ++p) THM_REQUIRE(nsub_of[p] > 0, "every problem needs at least one subdomain");
        for (int64_t k = 0; k < m->n_if; ++k)
            THM_REQUIRE(sp[m->if_recv[k]] == sp[m->if_send[k]], "subdomains of different problems share an interface");
        // global DOFs: each belongs to one problem, and the problems' DOFs form
        // contiguous increasing ranges (vertices numbered problem by problem)
        std::vector<int32_t> dp(m->n_dof, -1);
        for (int64_t c = 0; c < m->n_cell; ++c) {
            const int32_t p = sp[m->cell_sub[c]];
            for (int k = 0; k < m->dpc; ++k) {
                int32_t& q = dp[m->cell_dofs[c * m->dpc + k]];
                THM_REQUIRE(q < 0 || q == p, "problems share a DOF (the batch mesh must be a disjoint union)");
                q = p;
            }
        }
        std::vector<int64_t> dptr(n_prob + 1, 0), iptr(n_prob + 1, 0);
        for (int64_t d = 0; d < m->n_dof; ++d) {
            THM_REQUIRE(dp[d] >= 0 && (d == 0 || dp[d] >= dp[d - 1]),
                        "the problems' DOFs must form contiguous ranges (number the vertices problem by problem)");
            dptr[dp[d] + 1]++;
        }
        for (int64_t k = 0; k < m->n_if; ++k) iptr[sp[m->if_recv[k]] + 1]++;
        for (int p = 0; p < n_prob; ++p) { dptr[p + 1] += dptr[p]; iptr[p + 1] += iptr[p]; }
        std::vector<Chunk> ch;
        for (int p = 0; p < n_prob; ++p)
            for (int64_t b = dptr[p]; b < dptr[p + 1]; b += CHUNK) {
                Chunk c{};
                c.seg = p; c.begin = b; c.end = std::min<int64_t>(dptr[p + 1], b + CHUNK);
                ch.push_back(c);
            }
        m->n_prob = n_prob;
        m->sub_prob = sp;
        m->prob_dof_ptr = dptr;
        m->prob_if_ptr = iptr;
        m->dof_chunks = ch;
        m->d_dof_chunks.upload(ch);
        THM_CUDA(cudaDeviceSynchronize());
        return THM_OK;
    });
}

int thm_assemble_batch(thm_sys** out, const thm_mesh* m, const double* mu_inv, int mu_inv_on_device,
                       const double* omega, double kappa, const double* pol, const double* dir, void* stream) {
    if (!m || !omega) {
        set_last_error("NULL argument");
        if (out) *out = nullptr;
        return THM_EINVAL;
    }
    return assemble_common(out, m, mu_inv, mu_inv_on_device, std::vector<double>(omega, omega + m->n_prob), kappa,
                           pol, dir, stream);
}

int thm_ddm_solve(thm_sys* s, const thm_solve_opts* opts, double* u, thm_stats* stats) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && u, "NULL argument");
        return solve(s, opts, reinterpret_cast<double2*>(u), stats);
    });
}

int thm_ddm_solve_host(thm_sys* s, const thm_solve_opts* opts, double* u_host, thm_stats* stats) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && u_host, "NULL argument");
        DArr<double2> u;
        u.alloc(s->m->n_dof);
        int rc = solve(s, opts, u.p, stats);
        THM_CUDA(cudaMemcpyAsync(u_host, u.p, s->m->n_dof * sizeof(double2), cudaMemcpyDeviceToHost, s->st));
        THM_CUDA(cudaStreamSynchronize(s->st));
        return rc;
    });
}

int thm_adjoint(thm_sys* s, const thm_solve_opts* opts, const double* u, const double* dLdu_conj,
                double* grad_mu_inv, double* grad_omega, double* grad_kappa, thm_stats* stats) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && u && dLdu_conj && grad_mu_inv && grad_omega, "NULL argument");
        return adjoint(s, opts, reinterpret_cast<const double2*>(u), reinterpret_cast<const double2*>(dLdu_conj),
                       grad_mu_inv, grad_omega, grad_kappa, stats);
    });
}

void thm_sys_destroy(thm_sys* s) { delete s; }

int thm_sys_info(const thm_sys* s, int64_t* n_local, int64_t* n_iface, int32_t* n_sub, int64_t* nnz_stored) {
    return guarded([&]() -> int {
        THM_REQUIRE(s, "NULL system");
        if (n_local) *n_local = s->m->n_loc;
        if (n_iface) *n_iface = s->m->n_if;
        if (n_sub) *n_sub = s->m->n_sub;
        if (nnz_stored) *nnz_stored = s->m->n_slots;
        return THM_OK;
    });
}

int thm_local_dofs(const thm_sys* s, int64_t* gdof, int32_t* sub) {
    return guarded([&]() -> int {
        THM_REQUIRE(s, "NULL system");
        if (gdof) std::copy(s->m->loc_gdof.begin(), s->m->loc_gdof.end(), gdof);
        if (sub) std::copy(s->m->loc_sub.begin(), s->m->loc_sub.end(), sub);
        return THM_OK;
    });
}

int thm_iface_dofs(const thm_sys* s, int32_t* recv, int32_t* send, int64_t* gdof) {
    return guarded([&]() -> int {
        THM_REQUIRE(s, "NULL system");
        if (recv) std::copy(s->m->if_recv.begin(), s->m->if_recv.end(), recv);
        if (send) std::copy(s->m->if_send.begin(), s->m->if_send.end(), send);
        if (gdof) std::copy(s->m->if_gdof.begin(), s->m->if_gdof.end(), gdof);
        return THM_OK;
    });
}

int thm_apply_local(thm_sys* s, int op, int mode, const double* x, double* y) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && x && y, "NULL argument");
        apply_local(s, op, mode, reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(y));
        return THM_OK;
    });
}

int thm_sweep(thm_sys* s, const thm_solve_opts* opts, int with_sources, const double* g_in, double* g_out,
              double* u_loc, thm_stats* stats) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && u_loc, "NULL argument");
        THM_REQUIRE(s->m->n_if == 0 || (g_in && g_out), "NULL interface vector");
        return sweep_diag(s, opts, with_sources, reinterpret_cast<const double2*>(g_in),
                          reinterpret_cast<double2*>(g_out), reinterpret_cast<double2*>(u_loc), stats);
    });
}

int thm_local_sources(thm_sys* s, double* f_loc) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && f_loc, "NULL argument");
        THM_CUDA(cudaMemcpyAsync(f_loc, s->f_loc.p, s->m->n_loc * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
        THM_CUDA(cudaStreamSynchronize(s->st));
        return THM_OK;
    });
}

int thm_dirichlet_values(thm_sys* s, double* u_d) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && u_d, "NULL argument");
        THM_CUDA(cudaMemcpyAsync(u_d, s->uD.p, s->m->n_dof * sizeof(double2), cudaMemcpyDeviceToDevice, s->st));
        THM_CUDA(cudaStreamSynchronize(s->st));
        return THM_OK;
    });
}

int thm_alg_bytes(const thm_sys* s, int mode, int cls, double* bytes) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && bytes, "NULL argument");
        const thm_mesh* m = s->m;
        const double bv = mode == THM_MODE_MIXED ? 4.0 : 8.0;   // value
        const double bx = 2 * bv;                                // complex vector entry
        if (cls == THM_K_SPMV) {
            int64_t nnz = 0;
            for (uint8_t p : m->sell_pad) nnz += !p;
            *bytes = nnz * bv + 2.0 * m->n_loc * bv + 2.0 * m->n_loc * bx;
        } else if (cls == THM_K_PINV) {
            double w = 0, ne = 0, nb = 0;
            for (const auto& S : m->subs) {
                w += (double)bt_stream_values(S, m->levels.data());
                ne += (double)S.ne;
                nb += (double)(S.n - S.ne);
            }
            double tab = m->order == 2 ? (8 * ne + 12 * nb) : 0;
            *bytes = (w + tab) * bv + 2.0 * m->n_loc * bx;
        } else {
            fail(THM_EINVAL, "no byte model for this kernel class");
        }
        return THM_OK;
    });
}

int thm_work_bytes(const thm_sys* s, int mode, int cls, double* bytes) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && bytes, "NULL argument");
        THM_REQUIRE(cls == THM_K_PINV || cls == THM_K_SPMV || cls == THM_K_DOTS || cls == THM_K_UPDATE,
                    "no work counter for this kernel class");
        *bytes = 0;
        if (cls != THM_K_PINV) {
            if (!s->kwork.p) return THM_OK;
            std::vector<unsigned long long> h;
            s->kwork.download(h, s->st);
            const int o = mode == THM_MODE_MIXED ? 4 : 0;
            if (cls == THM_K_SPMV) {
                // rows processed x the SpMV byte model per row
                double full = 0;
                THM_REQUIRE(thm_alg_bytes(s, mode, THM_K_SPMV, &full) == THM_OK, "byte model");
                *bytes = full * (double)h[o] / (double)std::max<int64_t>(1, s->m->n_loc);
            } else {
                *bytes = (double)h[o + (cls == THM_K_DOTS ? 1 : 2)];
            }
            return THM_OK;
        }
        if (!s->bt_work.p) return THM_OK;
        std::vector<unsigned long long> h;
        s->bt_work.download(h, s->st);
        const bool f32 = mode == THM_MODE_MIXED;
        const double bv = f32 ? 4.0 : 8.0, bx = 2 * bv;
        const unsigned long long* c = h.data() + (f32 ? 2 : 0);
        *bytes = (double)c[0] * bv + 2.0 * (double)c[1] * bx;
        return THM_OK;
    });
}

int thm_factor_bytes(const thm_sys* s, int precond, int mode, double* bytes) {
    return guarded([&]() -> int {
        THM_REQUIRE(s && bytes, "NULL argument");
        THM_REQUIRE(precond == THM_PRECOND_BLOCKDIAG || precond == THM_PRECOND_FULL, "unknown preconditioner");
        const double bv = mode == THM_MODE_MIXED ? 4.0 : 8.0;
        *bytes = (double)s->m->fac_elems * bv * (precond == THM_PRECOND_FULL ? 2.0 : 1.0);
        return THM_OK;
    });
}

int64_t thm_kernel_launches(void) { return (int64_t)g_launches.load(); }

int thm_profile_enable(unsigned mask) {
    return guarded([&]() -> int {
        prof_set(mask);
        return THM_OK;
    });
}

int thm_profile_read(int cls, int64_t* launches, double* ms) {
    return guarded([&]() -> int {
        THM_REQUIRE(cls >= 0 && cls < THM_K_NCLASSES, "unknown kernel class");
        prof_read(cls, launches, ms);
        return THM_OK;
    });
}

}  // extern "C"

// Internal structures of the THM DDM-GMRES library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "thm.h"

namespace thm {

struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void set_last_error(const std::string& msg);

#define THM_CUDA(call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            ::thm::fail(e_ == cudaErrorMemoryAllocation ? THM_ENOMEM : THM_ECUDA,      \
                        std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)

#define THM_REQUIRE(cond, msg)                                                         \
    do {                                                                               \
        if (!(cond)) ::thm::fail(THM_EINVAL, msg);                                     \
    } while (0)

// Owning device array.
template <class T>
struct DArr {
    T* p = nullptr;
    size_t n = 0;
    DArr() = default;
    DArr(const DArr&) = delete;
    DArr& operator=(const DArr&) = delete;
    ~DArr() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) THM_CUDA(cudaMalloc(&p, count * sizeof(T)));
    }
    void zero(cudaStream_t st) {
        if (n) THM_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), st));
    }
    void upload(const std::vector<T>& h, cudaStream_t st = 0) {
        alloc(h.size());
        if (n) THM_CUDA(cudaMemcpyAsync(p, h.data(), n * sizeof(T), cudaMemcpyHostToDevice, st));
    }
    void download(std::vector<T>& h, cudaStream_t st = 0) const {
        h.resize(n);
        if (n) {
            THM_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, st));
            THM_CUDA(cudaStreamSynchronize(st));
        }
    }
};

void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st);
void prof_set(unsigned mask);
void prof_read(int cls, int64_t* launches, double* ms);

// Every kernel launch of the library goes through THM_LAUNCH (launch count,
// optional CUDA-event timing of its class).
#define THM_LAUNCH(cls, st, ...)            \
    do {                                    \
        ::thm::prof_begin((cls), (st));     \
        __VA_ARGS__;                        \
        ::thm::prof_end((cls), (st));       \
    } while (0)

constexpr int SELL_C = 32;       // rows per SELL slice (one warp)
constexpr int CHUNK = 1024;      // elements per reduction chunk of a segment

// One block of the level-block-tridiagonal factorisation of P_i.
struct Level {
    int32_t start;    // first local row (absolute index into local vectors)
    int32_t size;     // m_l
    int32_t prev;     // m_{l-1} (0 for the first level of a subdomain)
    int32_t next;     // m_{l+1} (0 for the last)
    int64_t offW;     // W_l = S_l^{-1}: m_l rows of stride r4(m_l) (16-byte aligned)
    int64_t offH;     // H_l^T, the backward-sweep product (l != kmid): H_l = W_l F_l above the
                      // middle level, W_l E_l below it; m_{l+1} resp. m_{l-1} rows of stride
                      // r4(m_l), or -1 (16-byte aligned)
    // coupling blocks of S to level l-1 (E) and l+1 (F): m_l+1 row pointers
    // (0-based, at cpl_ptr[eptr..]) and nz (column local to the neighbour
    // level, value) entries at cpl_col/cpl_val[eoff..]; offsets 16-byte aligned
    int64_t eptr, eoff, fptr, foff;
    int32_t enz, fnz;
};

struct Sub {
    int64_t off;      // first local row
    int64_t n;        // free DOFs
    int64_t ne;       // free edge DOFs (rows off .. off+ne-1); cell bubbles follow
    int32_t lev0;     // first level
    int32_t nlev;
    int32_t kmid;     // middle level of the twisted factorisation (0 <= kmid < nlev)
    int32_t cell0;    // order 2: slot of the first bubble cell (rows off+ne.. in groups of 4) in thm_sys::tab_e8
};

// Values one block solve streams for subdomain S (the byte model of the
// block-solve kernel, in values): W_l once for every level (forward steps and
// the middle level), H_l for every level but the middle (backward steps),
// and the coupling lists of the forward and middle steps (E_1..E_k of the top
// chain, F_k..F_{L-2} of the bottom one).
inline int64_t bt_stream_values(const Sub& S, const Level* lv) {
    int64_t w = 0;
    for (int l = 0; l < S.nlev; ++l) {
        const Level& L = lv[S.lev0 + l];
        w += (int64_t)L.size * L.size;
        if (l != S.kmid) w += (int64_t)L.size * (l < S.kmid ? L.next : L.prev);
        if (l >= 1 && l <= S.kmid) w += L.enz;
        if (l >= S.kmid && l + 1 < S.nlev) w += L.fnz;
    }
    return w;
}

// A contiguous piece of one segment, used for deterministic segmented reductions.
struct Chunk {
    int32_t seg;
    int32_t pad;
    int64_t begin;
    int64_t end;
};

}  // namespace thm

struct thm_mesh {
    int dim = 0, order = 0, dpc = 0, epc = 0, max_block = 0;
    int64_t n_vert = 0, n_cell = 0, n_bface = 0, n_edge = 0, n_dof = 0;
    int n_sub = 0;
    std::vector<double> coords;
    std::vector<int64_t> cells;
    std::vector<int32_t> cell_sub;
    std::vector<int64_t> bfaces;
    std::vector<uint8_t> btag;
    std::vector<int64_t> edge_lo, edge_hi;          // sorted (lo, hi)
    std::vector<int64_t> cell_dofs;                 // [n_cell][dpc]
    std::vector<int8_t> cell_signs;                 // [n_cell][dpc]
    std::vector<uint8_t> is_dir;                    // [n_dof]
    std::vector<int64_t> dir_edges;                 // edges carrying Dirichlet DOFs
    std::vector<int64_t> dir_dofs;                  // Dirichlet DOFs, increasing
    thm::DArr<int64_t> d_dir_dofs;

    // local (per-subdomain, free DOFs) structure
    int64_t n_loc = 0;
    int64_t n_bcell = 0;                            // order 2: cells (bubble groups) over all subdomains
    std::vector<thm::Sub> subs;
    std::vector<int64_t> loc_gdof;                  // [n_loc]
    std::vector<int32_t> loc_sub;                   // [n_loc]
    std::vector<int32_t> cell_loc;                  // [n_cell][dpc] local row or -1
    // SELL-32 pattern of P_i (all subdomains), columns are local indices
    int64_t n_slices = 0, n_slots = 0;
    std::vector<int64_t> slice_ptr;                 // [n_slices+1]
    std::vector<int32_t> sell_col;                  // [n_slots]; padding = own row
    // the same columns relative to the row's subdomain (col - off of the
    // row's subdomain) in 16 bits, for the SpMV, when every subdomain has at
    // most 65,536 local DOFs (col16); the factorisation keeps sell_col
    std::vector<uint16_t> sell_col16;
    bool col16 = false;
    std::vector<uint8_t> sell_pad;                  // [n_slots] 1 = padding
    // assembly plan: cells holding each local row (ascending), <= maxc
    int maxc = 0;
    std::vector<int32_t> row_cell, row_k;           // [n_loc][maxc]
    // faces with impedance (kind 1, Gamma^inf) or transmission (kind 2, Sigma)
    // terms; fd DOFs per face (2-D order 1: 1, order 2: 2, 3-D: 4)
    static constexpr int RF = 4;                     // faces per local row, at most
    int fd = 0;
    int64_t n_face = 0;
    std::vector<int32_t> face_v;                    // [n_face][4] vertices, face-local tensor order
    std::vector<int32_t> face_dof;                  // [n_face][fd]
    std::vector<int8_t> face_sgn;                   // [n_face][fd]
    std::vector<int8_t> face_kind;                  // [n_face]
    std::vector<int32_t> face_sub;                  // [n_face][2] subdomains (-1: none)
    std::vector<int32_t> face_loc;                  // [n_face][2][fd] local rows per side (-1: Dirichlet)
    std::vector<int32_t> row_face;                  // [n_loc][RF] face ids (-1: none)
    std::vector<int8_t> row_face_a, row_face_side;  // [n_loc][RF]
    // levels of the block-tridiagonal factorisation
    std::vector<thm::Level> levels;
    int max_m = 0;
    int max_lev = 0;                                // most levels of a subdomain
    int64_t bt_nvec = 0;                            // longest half-chain vector of the twisted solve
    std::vector<int64_t> bt_welem;                  // [n_sub] values one block solve reads (W, couplings, tables)
    thm::DArr<int64_t> d_bt_welem;
    int64_t fac_elems = 0;
    // W-tile size of the block-solve kernel picked by its autotuner ([0] FP64
    // factors, [1] FP32), 0 until the first apply of a system on this mesh.
    // The factor layout (levels, block sizes) is the mesh's, so every system
    // assembled on the mesh reuses the choice.
    mutable size_t bt_tile[4] = {0, 0, 0, 0};    // [2], [3]: complex factors (full-block preconditioner)
    // level couplings of S as compact CSR lists (columns local to the
    // neighbouring level; slot = position of the value in the SELL arrays)
    std::vector<int32_t> cpl_ptr, cpl_col;
    std::vector<int64_t> cpl_slot;                  // -1 for alignment padding
    int max_cnz = 0;                                // largest coupling block
    int64_t max_ne = 0;                             // largest number of edge DOFs of a subdomain
    // reduction chunks over subdomains
    std::vector<thm::Chunk> chunks;
    // interface entries (directed pairs i <- j, one per free DOF on Sigma_ij)
    int64_t n_if = 0;
    std::vector<int32_t> if_recv, if_send, if_rowi, if_partner;
    std::vector<int64_t> if_gdof;
    // terms of (M_Sigma_ij u_j)[g] per entry: face, a, b, sender column (-(gdof+1): Dirichlet)
    std::vector<int64_t> if_ptr;
    std::vector<int32_t> if_tf, if_tcol;
    std::vector<int8_t> if_ta, if_tb;
    std::vector<int64_t> rowg_ptr;                  // [n_loc+1] local row -> entries received
    std::vector<int32_t> rowg_idx;
    // independent problems sharing the mesh (a batch): subdomain -> problem,
    // each problem's contiguous range of global DOFs and of interface entries,
    // and reduction chunks over the global DOFs segmented by problem
    int n_prob = 1;
    mutable bool assembled = false;                 // a system was built on this mesh
    std::vector<int32_t> sub_prob;                  // [n_sub]
    std::vector<int64_t> prob_dof_ptr, prob_if_ptr; // [n_prob+1]
    std::vector<thm::Chunk> dof_chunks;
    // global <-> local
    std::vector<int32_t> owner_loc;                 // [n_dof] lowest-subdomain copy, -1 Dirichlet
    std::vector<int64_t> copy_ptr;                  // [n_dof+1]
    std::vector<int32_t> copy_idx;
    std::vector<uint8_t> loc_is_owner;              // [n_loc]
    std::vector<uint8_t> loc_is_bub;                // [n_loc] order-2 cell bubble

    // device mirrors
    thm::DArr<double> d_coords;
    thm::DArr<int32_t> d_cells, d_cell_dofs, d_cell_loc, d_sell_col, d_row_cell, d_row_k;
    thm::DArr<uint16_t> d_sell_col16;
    thm::DArr<int64_t> d_edge_lo, d_edge_hi, d_slice_ptr, d_dir_edges, d_loc_gdof, d_rowg_ptr,
        d_copy_ptr;
    thm::DArr<int8_t> d_cell_signs, d_face_sgn, d_face_kind, d_row_face_a, d_row_face_side, d_if_ta, d_if_tb;
    thm::DArr<uint8_t> d_sell_pad, d_loc_is_owner, d_loc_is_bub;
    thm::DArr<int32_t> d_if_rowi, d_if_partner, d_rowg_idx, d_owner_loc, d_copy_idx, d_loc_sub, d_face_v,
        d_face_dof, d_face_loc, d_row_face, d_if_tf, d_if_tcol;
    thm::DArr<int64_t> d_if_ptr;
    thm::DArr<thm::Level> d_levels;
    thm::DArr<int32_t> d_cpl_ptr, d_cpl_col;
    thm::DArr<int64_t> d_cpl_slot;
    thm::DArr<thm::Sub> d_subs;
    thm::DArr<thm::Chunk> d_chunks;
    thm::DArr<thm::Chunk> d_dof_chunks;
};

namespace thm { struct Work; }

// Assembled system of one (mesh, mu^{-1}, omega, kappa, E^inc).
struct thm_sys {
    const thm_mesh* m = nullptr;
    cudaStream_t st = 0;
    double omega = 0, kappa = 0;       // omega: the first problem's (the only one unless batched)
    std::vector<double> omega_prob;    // [n_prob]
    thm::DArr<double> w2c;             // [n_cell] omega^2 of the cell's problem
    thm::DArr<double> kwf;             // [n_face] kappa*omega of the face's problem
    thm::DArr<double> omd;             // [n_dir_edges] omega of the Dirichlet edge's problem
    double pol[6] = {0};   // complex [dim]
    double dir[3] = {0};
    thm::DArr<double> mu_inv;          // [n_cell]
    thm::DArr<double> ref;             // reference matrices (see assemble.cu)
    thm::DArr<double> val64;           // SELL values of P_i = Re(T_i), FP64
    thm::DArr<float> val32;            // same, FP32
    // transmission coefficient on Sigma_ij in units of kappa*omega: (0, 1) is
    // i kappa omega, the impedance condition of Eq. 5; a real part adds
    // trans_re * kappa omega M_Sigma to Re(T_i) (and then K_i^loc, which has no
    // Sigma terms, gets value arrays of its own)
    double trans_re = 0.0, trans_im = 1.0;
    thm::DArr<double> valK64;          // SELL values of Re(K_i^loc) when trans_re != 0
    thm::DArr<float> valK32;
    const double* kloc_val64() const { return valK64.p ? valK64.p : val64.p; }
    const float* kloc_val32() const { return valK32.p ? valK32.p : val32.p; }
    thm::DArr<double> eps;             // [n_cell] relative permittivity (mass-term weight), 1 if not given
    thm::DArr<double> bg64, bs64;      // kappa*omega * diagonal face masses: Gamma^inf, Sigma
    thm::DArr<float> bg32, bs32;
    thm::DArr<double> if_val;          // values of the interface-entry terms (face masses)
    thm::DArr<double> bvg64, bvs64;    // 3-D: kappa*omega face masses on the SELL pattern (Gamma^inf, Sigma)
    thm::DArr<float> bvg32, bvs32;
    thm::DArr<double2> uD;             // [n_dof] Dirichlet values
    // Dirichlet values given by the caller (thm_assemble_dirichlet) instead of
    // the moments of a plane wave: [n_dir] in increasing global-DOF order
    bool dir_user = false;
    thm::DArr<double2> dir_vals;
    thm::DArr<double2> f_loc;          // [n_loc] subdomain sources: -(T_i)_{F,D} u_D (Eq. 5)
    thm::DArr<double2> f_res;          // [n_loc] split of the global right-hand side: -(K_i^loc)_{F,D} u_D
    // block-tridiagonal factors of P_i (lazily built per precision)
    bool fac64_ok = false, fac32_ok = false;
    thm::DArr<double> fac64;
    thm::DArr<float> fac32;
    // complex factors of the full 2x2 block operator (Section 3.2's
    // alternative preconditioner), lazily built per precision
    bool facc64_ok = false, facc32_ok = false;
    thm::DArr<double2> facc64;
    thm::DArr<float2> facc32;
    // static condensation of order-2 cell bubbles: S = P_EE - P_EI D^{-1} P_IE
    thm::DArr<double> sval64;          // SELL values of S on edge rows/columns (P elsewhere 0)
    thm::DArr<float> sval32;
    thm::DArr<double> cinv64, cg64;    // per cell: D_II^{-1} (4x4), G = P_EI D_II^{-1} (8x4)
    thm::DArr<float> cinv32, cg32;
    thm::DArr<int> dev_err;            // set by a device-side bounded wait that gave up
    thm::DArr<double> cpl64;           // values of the level coupling lists
    thm::DArr<float> cpl32;
    // order-2 gather tables (structure of arrays, [8][n_loc]): for an edge row
    // the <= 8 (bubble, G entry) pairs of r_E - G r_I; for a bubble row the 4
    // (bubble, D^{-1} entry) and 8 (edge, -G entry) pairs of D^{-1} r_I - G^T x_E.
    // The bubbles of a cell are 4 consecutive local rows, so the indices are
    // not stored per entry: tab_ab [2][n_loc] holds an edge row's (<= 2) cells'
    // first bubble rows (-1: none; entry u*4+k of av belongs to bubble ab[u]+k),
    // tab_e8 [bubble cells][8] a cell's 8 edge rows (-1: Dirichlet), the cell of
    // bubble row b being slot subs.cell0 + (b - off - ne) / 4
    thm::DArr<int32_t> tab_ab, tab_e8;
    thm::DArr<double> tab_av64, tab_cv64, tab_ev64;
    thm::DArr<float> tab_av32, tab_cv32, tab_ev32;
    // block-solve work actually done, per factor precision ([0..1] FP64, [2..3]
    // FP32): values read and local rows processed, summed by the kernel over
    // the subdomains it did not skip
    mutable thm::DArr<unsigned long long> bt_work;
    // work counters of the SpMV and Gram-Schmidt kernels, [8]: (FP32 ? 4 : 0)
    // + 0 SpMV rows processed, 1 dot-product pass bytes, 2 update pass bytes
    mutable thm::DArr<unsigned long long> kwork;
    // solver workspace (allocated on first solve, see solve.cu)
    thm::Work* w = nullptr;
    ~thm_sys();
};

namespace thm {
void build_mesh(thm_mesh* m);
void assemble(thm_sys* s);
void ensure_factor(thm_sys* s, bool fp32);
void ensure_factor_full(thm_sys* s, bool fp32);
}  // namespace thm

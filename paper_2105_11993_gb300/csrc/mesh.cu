// Mesh numbering, orientation signs and the subdomain structure (Section 2:
// the space N_h^p; Section 3.1: the partition into Omega_i and Sigma_ij).
#include <algorithm>
#include <array>
#include <tuple>
#include <cmath>
#include <numeric>
#include <queue>

#include "common.cuh"

namespace thm {

// Local edges of a tensor-order quad / hex: (a -> b) along +xi, +eta, +zeta.
__constant__ int c_edges2[4][2] = {{0, 1}, {2, 3}, {0, 2}, {1, 3}};
__constant__ int c_edges3[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3},
                                    {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
static const int h_edges2[4][2] = {{0, 1}, {2, 3}, {0, 2}, {1, 3}};
static const int h_edges3[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3},
                                    {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};

// Edge id of (a, b) by binary search in the lexicographically sorted table.
__device__ __forceinline__ int64_t find_edge(const int64_t* lo, const int64_t* hi, int64_t n,
                                             int64_t a, int64_t b) {
    int64_t x = a < b ? a : b, y = a < b ? b : a;
    int64_t l = 0, r = n - 1;
    while (l <= r) {
        int64_t mid = (l + r) >> 1;
        int64_t ml = lo[mid], mh = hi[mid];
        if (ml == x && mh == y) return mid;
        if (ml < x || (ml == x && mh < y)) l = mid + 1;
        else r = mid - 1;
    }
    return -1;
}

// DOF ids and orientation signs of every cell.  Whitney DOF of a local edge
// (a -> b) has sign +1 iff id(a) < id(b); order-2 gradient and bubble DOFs
// carry no sign.
__global__ void k_cell_dofs(int dim, int order, int64_t n_cell, const int32_t* __restrict__ cells,
                            const int64_t* __restrict__ elo, const int64_t* __restrict__ ehi,
                            int64_t n_edge, int32_t* __restrict__ dofs, int8_t* __restrict__ signs,
                            int* __restrict__ bad) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_cell) return;
    const int nv = dim == 2 ? 4 : 8;
    const int ne = dim == 2 ? 4 : 12;
    const int dpc = (order == 1) ? ne : 12;
    const int32_t* cv = cells + c * nv;
    for (int k = 0; k < ne; ++k) {
        int a = dim == 2 ? c_edges2[k][0] : c_edges3[k][0];
        int b = dim == 2 ? c_edges2[k][1] : c_edges3[k][1];
        int64_t va = cv[a], vb = cv[b];
        int64_t e = find_edge(elo, ehi, n_edge, va, vb);
        if (e < 0) { atomicExch(bad, 1); e = 0; }
        int8_t s = va < vb ? 1 : -1;
        if (order == 1) {
            dofs[c * dpc + k] = (int32_t)e;
            signs[c * dpc + k] = s;
        } else {
            dofs[c * dpc + 2 * k] = (int32_t)(2 * e);
            signs[c * dpc + 2 * k] = s;
            dofs[c * dpc + 2 * k + 1] = (int32_t)(2 * e + 1);
            signs[c * dpc + 2 * k + 1] = 1;
        }
    }
    if (order == 2) {
        for (int k = 0; k < 4; ++k) {
            dofs[c * dpc + 8 + k] = (int32_t)(2 * n_edge + 4 * c + k);
            signs[c * dpc + 8 + k] = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Global edges on the device: every (cell, local edge) gives the key
// min(id) * n_vert + max(id); the distinct keys in increasing order are the
// edges in the lexicographic order of (min id, max id).  A stable LSD radix
// sort (8-bit digits, 256-key tiles) orders the keys, then the first key of
// each run of equal keys is kept.  Everything is deterministic.
// ---------------------------------------------------------------------------
constexpr int RX_TILE = 256;                      // keys per tile (one per thread)
constexpr int RX_BINS = 256;                      // 8-bit digits

__global__ void k_edge_keys(int dim, int64_t n_cell, const int32_t* __restrict__ cells, int64_t n_vert,
                            unsigned long long* __restrict__ keys) {
    const int ne = dim == 2 ? 4 : 12, nv = dim == 2 ? 4 : 8;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_cell * ne) return;
    const int64_t c = i / ne;
    const int k = (int)(i % ne);
    const int a = dim == 2 ? c_edges2[k][0] : c_edges3[k][0];
    const int b = dim == 2 ? c_edges2[k][1] : c_edges3[k][1];
    const int64_t va = cells[c * nv + a], vb = cells[c * nv + b];
    const int64_t lo = va < vb ? va : vb, hi = va < vb ? vb : va;
    keys[i] = (unsigned long long)lo * (unsigned long long)n_vert + (unsigned long long)hi;
}

// Per tile and warp: how many keys of each digit precede a key in its warp
// (match mask), the warp's count per digit, and the tile's count per digit.
__device__ __forceinline__ void rx_rank(unsigned digit, bool valid, int* wcnt /* [8][256] */, int& rank_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? digit : 0xffffffffu) & vmask;
    rank_w = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank_w == 0) wcnt[warp * RX_BINS + digit] = __popc(peers);
}

// Tile histogram of the digit at `shift`: hist[bin * n_tiles + tile].
__global__ void __launch_bounds__(RX_TILE) k_rx_hist(int64_t n, const unsigned long long* __restrict__ keys,
                                                     int shift, int n_tiles, unsigned* __restrict__ hist) {
    __shared__ int wcnt[RX_TILE / 32 * RX_BINS];
    for (int t = threadIdx.x; t < RX_TILE / 32 * RX_BINS; t += blockDim.x) wcnt[t] = 0;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)RX_TILE + threadIdx.x;
    const bool valid = i < n;
    const unsigned d = valid ? (unsigned)((keys[i] >> shift) & (RX_BINS - 1)) : 0u;
    int r;
    rx_rank(d, valid, wcnt, r);
    __syncthreads();
    int sum = 0;
    for (int w = 0; w < RX_TILE / 32; ++w) sum += wcnt[w * RX_BINS + threadIdx.x];
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = (unsigned)sum;
}

// Stable scatter: position = offs[bin * n_tiles + tile] (exclusive scan of
// the histograms, bin major) + the counts of earlier warps + the rank in the warp.
__global__ void __launch_bounds__(RX_TILE) k_rx_scatter(int64_t n, const unsigned long long* __restrict__ in,
                                                        int shift, int n_tiles, const unsigned* __restrict__ offs,
                                                        unsigned long long* __restrict__ out) {
    __shared__ int wcnt[RX_TILE / 32 * RX_BINS];
    for (int t = threadIdx.x; t < RX_TILE / 32 * RX_BINS; t += blockDim.x) wcnt[t] = 0;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)RX_TILE + threadIdx.x;
    const bool valid = i < n;
    const unsigned long long key = valid ? in[i] : 0ull;
    const unsigned d = (unsigned)((key >> shift) & (RX_BINS - 1));
    int r;
    rx_rank(d, valid, wcnt, r);
    __syncthreads();
    if (!valid) return;
    const int warp = threadIdx.x >> 5;
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wcnt[w * RX_BINS + d];
    out[offs[(int64_t)d * n_tiles + blockIdx.x] + before + r] = key;
}

// Exclusive scan of n unsigned values in place (three passes over blocks of
// 1024 values; deterministic).
__global__ void k_scan_block_sums(int64_t n, const unsigned* __restrict__ a, unsigned* __restrict__ sums) {
    __shared__ unsigned sw[32];
    unsigned s = 0;
    for (int64_t i = blockIdx.x * 1024ll + threadIdx.x; i < n && i < (blockIdx.x + 1) * 1024ll; i += blockDim.x) s += a[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sw[q];
        sums[blockIdx.x] = t;
    }
}
__global__ void k_scan_sums_serial(int nb, unsigned* __restrict__ sums) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned run = 0;
    for (int b = 0; b < nb; ++b) {
        const unsigned v = sums[b];
        sums[b] = run;
        run += v;
    }
}
// one block of 1024 threads per 1024 values: block-local exclusive scan plus the block offset
__global__ void __launch_bounds__(1024) k_scan_apply(int64_t n, unsigned* __restrict__ a,
                                                     const unsigned* __restrict__ sums) {
    __shared__ unsigned sw[32];
    const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    const unsigned v = i < n ? a[i] : 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sw[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned x = sw[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        sw[lane] = x;                              // inclusive over warps
    }
    __syncthreads();
    const unsigned warp_off = warp > 0 ? sw[warp - 1] : 0u;
    if (i < n) a[i] = sums[blockIdx.x] + warp_off + incl - v;
}

static void device_exclusive_scan(unsigned* a, int64_t n, DArr<unsigned>& sums) {
    const int64_t nb = (n + 1023) / 1024;
    if ((int64_t)sums.n < nb) sums.alloc(nb);
    THM_LAUNCH(THM_K_SETUP, 0, k_scan_block_sums<<<(unsigned)nb, 256>>>(n, a, sums.p));
    THM_LAUNCH(THM_K_SETUP, 0, k_scan_sums_serial<<<1, 32>>>((int)nb, sums.p));
    THM_LAUNCH(THM_K_SETUP, 0, k_scan_apply<<<(unsigned)nb, 1024>>>(n, a, sums.p));
}

// flag[i] = 1 for the first key of each run of equal keys
__global__ void k_run_heads(int64_t n, const unsigned long long* __restrict__ keys, unsigned* __restrict__ flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}
__global__ void k_edges_from_keys(int64_t n, const unsigned long long* __restrict__ keys,
                                  const unsigned* __restrict__ pos, int64_t n_vert, int64_t* __restrict__ elo,
                                  int64_t* __restrict__ ehi) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !(i == 0 || keys[i] != keys[i - 1])) return;
    const unsigned long long k = keys[i];
    elo[pos[i]] = (int64_t)(k / (unsigned long long)n_vert);
    ehi[pos[i]] = (int64_t)(k % (unsigned long long)n_vert);
}

// The distinct edges (lexicographic (lo, hi)) of the cells, computed on the
// device into m->d_edge_lo / d_edge_hi and copied to the host tables.
static void device_edges(thm_mesh* m) {
    const int ne = m->dim == 2 ? 4 : 12;
    const int64_t n = m->n_cell * ne;
    THM_REQUIRE(n < (int64_t)UINT32_MAX, "too many cell edges");
    DArr<unsigned long long> ka, kb;
    ka.alloc(n);
    kb.alloc(n);
    const int th = 256;
    auto grid = [&](int64_t c) { return (unsigned)((c + th - 1) / th); };
    THM_LAUNCH(THM_K_SETUP, 0, k_edge_keys<<<grid(n), th>>>(m->dim, m->n_cell, m->d_cells.p, m->n_vert, ka.p));
    // digits needed for keys < n_vert^2
    const unsigned long long kmax = (unsigned long long)m->n_vert * (unsigned long long)m->n_vert;
    int bits = 1;
    while (bits < 64 && (kmax >> bits) != 0) ++bits;
    const int n_tiles = (int)((n + RX_TILE - 1) / RX_TILE);
    DArr<unsigned> hist, sums;
    hist.alloc((size_t)RX_BINS * n_tiles);
    unsigned long long* src = ka.p;
    unsigned long long* dst = kb.p;
    for (int shift = 0; shift < bits; shift += 8) {
        THM_LAUNCH(THM_K_SETUP, 0, k_rx_hist<<<n_tiles, RX_TILE>>>(n, src, shift, n_tiles, hist.p));
        device_exclusive_scan(hist.p, (int64_t)RX_BINS * n_tiles, sums);
        THM_LAUNCH(THM_K_SETUP, 0, k_rx_scatter<<<n_tiles, RX_TILE>>>(n, src, shift, n_tiles, hist.p, dst));
        std::swap(src, dst);
    }
    DArr<unsigned> pos;
    pos.alloc(n);
    THM_LAUNCH(THM_K_SETUP, 0, k_run_heads<<<grid(n), th>>>(n, src, pos.p));
    unsigned last_flag = 0, last_pos = 0;
    THM_CUDA(cudaMemcpy(&last_flag, pos.p + (n - 1), sizeof(unsigned), cudaMemcpyDeviceToHost));
    device_exclusive_scan(pos.p, n, sums);
    THM_CUDA(cudaMemcpy(&last_pos, pos.p + (n - 1), sizeof(unsigned), cudaMemcpyDeviceToHost));
    m->n_edge = (int64_t)last_pos + last_flag;
    m->d_edge_lo.alloc(m->n_edge);
    m->d_edge_hi.alloc(m->n_edge);
    THM_LAUNCH(THM_K_SETUP, 0, k_edges_from_keys<<<grid(n), th>>>(n, src, pos.p, m->n_vert, m->d_edge_lo.p,
                                                                  m->d_edge_hi.p));
    THM_CUDA(cudaGetLastError());
    m->d_edge_lo.download(m->edge_lo);
    m->d_edge_hi.download(m->edge_hi);
}

static int64_t host_find_edge(const thm_mesh* m, int64_t a, int64_t b) {
    int64_t x = std::min(a, b), y = std::max(a, b);
    auto it = std::lower_bound(m->edge_lo.begin(), m->edge_lo.end(), x);
    int64_t i0 = it - m->edge_lo.begin();
    auto it2 = std::upper_bound(m->edge_lo.begin(), m->edge_lo.end(), x);
    int64_t i1 = it2 - m->edge_lo.begin();
    auto jt = std::lower_bound(m->edge_hi.begin() + i0, m->edge_hi.begin() + i1, y);
    int64_t j = jt - m->edge_hi.begin();
    if (j < i1 && m->edge_hi[j] == y) return j;
    return -1;
}

static void check_axis_aligned(const thm_mesh* m) {
    const int d = m->dim, nv = d == 2 ? 4 : 8;
    for (int64_t c = 0; c < m->n_cell; ++c) {
        const int64_t* cv = &m->cells[c * nv];
        auto X = [&](int v, int k) { return m->coords[cv[v] * d + k]; };
        double ax[3][3];
        int axes = d;
        int corner[3] = {1, 2, 4};
        for (int a = 0; a < axes; ++a)
            for (int k = 0; k < d; ++k) ax[a][k] = X(corner[a], k) - X(0, k);
        double len[3];
        for (int a = 0; a < axes; ++a) {
            len[a] = 0;
            int nz = 0;
            for (int k = 0; k < d; ++k) {
                len[a] += ax[a][k] * ax[a][k];
                nz += ax[a][k] != 0.0;
            }
            len[a] = std::sqrt(len[a]);
            THM_REQUIRE(nz == 1 && len[a] > 0, "cell " + std::to_string(c) + " is not axis-aligned");
        }
        // every corner = v0 + sum of the selected axis vectors
        for (int v = 0; v < nv; ++v)
            for (int k = 0; k < d; ++k) {
                double x = X(0, k);
                for (int a = 0; a < axes; ++a)
                    if ((v >> a) & 1) x += ax[a][k];
                THM_REQUIRE(std::fabs(x - X(v, k)) <= 1e-12 * (len[0] + std::fabs(x)),
                            "cell " + std::to_string(c) + " is not a tensor-order box");
            }
    }
}

void build_mesh(thm_mesh* m) {
    const int d = m->dim, nv = d == 2 ? 4 : 8;
    const int ne = d == 2 ? 4 : 12;
    m->epc = ne;
    m->dpc = (m->order == 1) ? ne : 12;
    check_axis_aligned(m);

    // ---- global edges: distinct (lo, hi) pairs in lexicographic order (device sort)
    std::vector<int32_t> cells32(m->cells.begin(), m->cells.end());
    m->d_cells.upload(cells32);
    m->d_coords.upload(m->coords);
    device_edges(m);
    m->n_dof = m->order == 1 ? m->n_edge : 2 * m->n_edge + 4 * m->n_cell;
    THM_REQUIRE(m->n_dof < (int64_t)INT32_MAX, "more than 2^31 DOFs");

    // ---- per-cell DOFs and signs on the device
    m->d_cell_dofs.alloc(m->n_cell * m->dpc);
    m->d_cell_signs.alloc(m->n_cell * m->dpc);
    DArr<int> bad;
    bad.alloc(1);
    bad.zero(0);
    int th = 256;
    THM_LAUNCH(THM_K_SETUP, 0, k_cell_dofs<<<(unsigned)((m->n_cell + th - 1) / th), th>>>(
        d, m->order, m->n_cell, m->d_cells.p, m->d_edge_lo.p, m->d_edge_hi.p, m->n_edge,
        m->d_cell_dofs.p, m->d_cell_signs.p, bad.p));
    THM_CUDA(cudaGetLastError());
    std::vector<int> hbad;
    bad.download(hbad);
    THM_REQUIRE(hbad[0] == 0, "internal: edge lookup failed");
    std::vector<int32_t> cd32;
    m->d_cell_dofs.download(cd32);
    m->cell_dofs.assign(cd32.begin(), cd32.end());
    m->d_cell_signs.download(m->cell_signs);
    const int dpc = m->dpc;

    // ---- edge -> cells (first two) and edge of each (cell, local edge)
    std::vector<int32_t> ecell(m->n_edge * 2, -1);
    auto edge_of = [&](int64_t c, int k) -> int64_t {
        int64_t dof = m->cell_dofs[c * dpc + (m->order == 1 ? k : 2 * k)];
        return m->order == 1 ? dof : dof / 2;
    };
    if (d == 2) {
        for (int64_t c = 0; c < m->n_cell; ++c)
            for (int k = 0; k < ne; ++k) {
                int64_t e = edge_of(c, k);
                if (ecell[2 * e] < 0) ecell[2 * e] = (int32_t)c;
                else ecell[2 * e + 1] = (int32_t)c;
            }
    }

    // ---- boundary faces: Dirichlet DOFs and impedance edges
    m->is_dir.assign(m->n_dof, 0);
    std::vector<int8_t> edge_kind(m->n_edge, 0);   // 1 = Gamma^inf face edge (2-D)
    const int fv = d == 2 ? 2 : 4;
    for (int64_t f = 0; f < m->n_bface; ++f) {
        const int64_t* v = &m->bfaces[f * fv];
        for (int k = 0; k < fv; ++k)
            THM_REQUIRE(v[k] >= 0 && v[k] < m->n_vert, "bface vertex out of range");
        std::vector<int64_t> es;
        if (d == 2) {
            es.push_back(host_find_edge(m, v[0], v[1]));
        } else {
            for (int k = 0; k < 4; ++k) es.push_back(host_find_edge(m, v[h_edges2[k][0]], v[h_edges2[k][1]]));
        }
        for (int64_t e : es) THM_REQUIRE(e >= 0, "bface " + std::to_string(f) + " is not a cell face");
        if (d == 2) THM_REQUIRE(ecell[2 * es[0] + 1] < 0, "bface " + std::to_string(f) + " is interior");
        if (m->btag[f] == THM_TAG_DIRICHLET) {
            for (int64_t e : es) {
                if (m->order == 1) m->is_dir[e] = 1;
                else { m->is_dir[2 * e] = 1; m->is_dir[2 * e + 1] = 1; }
                m->dir_edges.push_back(e);
            }
        } else if (m->btag[f] == THM_TAG_IMPEDANCE) {
            if (d == 2) edge_kind[es[0]] = 1;
        } else {
            THM_REQUIRE(m->btag[f] == THM_TAG_NATURAL, "unknown boundary tag");
        }
    }
    std::sort(m->dir_edges.begin(), m->dir_edges.end());
    m->dir_edges.erase(std::unique(m->dir_edges.begin(), m->dir_edges.end()), m->dir_edges.end());

    // ---- subdomains
    const int ns = m->n_sub;
    std::vector<std::vector<int64_t>> sub_cells(ns);
    for (int64_t c = 0; c < m->n_cell; ++c) sub_cells[m->cell_sub[c]].push_back(c);
    for (int s = 0; s < ns; ++s) THM_REQUIRE(!sub_cells[s].empty(), "empty subdomain " + std::to_string(s));

    // DOF "position" along the sweep axis (last coordinate): edge midpoint or cell centre
    auto dof_pos = [&](int64_t c, int k) -> double {
        int64_t dof = m->cell_dofs[c * dpc + k];
        if (m->order == 2 && k >= 8) {
            double y = 0;
            for (int v = 0; v < nv; ++v) y += m->coords[m->cells[c * nv + v] * d + d - 1];
            return y / nv;
        }
        int64_t e = m->order == 1 ? dof : dof / 2;
        return 0.5 * (m->coords[m->edge_lo[e] * d + d - 1] + m->coords[m->edge_hi[e] * d + d - 1]);
    };

    m->cell_loc.assign(m->n_cell * dpc, -1);
    m->subs.resize(ns);
    m->loc_gdof.clear();
    m->loc_sub.clear();
    m->levels.clear();
    m->n_bcell = 0;
    std::vector<std::vector<int32_t>> row_cols_all;   // per local row: sorted local columns
    m->maxc = d == 2 ? 2 : 4;
    std::vector<int32_t> row_cell_v, row_k_v;
    int64_t off = 0;
    for (int s = 0; s < ns; ++s) {
        const auto& cs = sub_cells[s];
        // free DOFs of the subdomain
        std::vector<int64_t> gd;
        for (int64_t c : cs)
            for (int k = 0; k < dpc; ++k) {
                int64_t g = m->cell_dofs[c * dpc + k];
                if (!m->is_dir[g]) gd.push_back(g);
            }
        std::sort(gd.begin(), gd.end());
        gd.erase(std::unique(gd.begin(), gd.end()), gd.end());
        const int64_t n = (int64_t)gd.size();
        THM_REQUIRE(n > 0, "subdomain without free DOFs");
        auto lid = [&](int64_t g) { return (int64_t)(std::lower_bound(gd.begin(), gd.end(), g) - gd.begin()); };
        // adjacency through cells, cells of each DOF, position
        std::vector<std::vector<int32_t>> adj(n);
        std::vector<std::vector<std::pair<int32_t, int32_t>>> dcells(n);
        std::vector<double> pos(n, 0.0);
        for (int64_t c : cs) {
            int32_t loc[12];
            for (int k = 0; k < dpc; ++k) {
                int64_t g = m->cell_dofs[c * dpc + k];
                loc[k] = m->is_dir[g] ? -1 : (int32_t)lid(g);
                if (loc[k] >= 0) {
                    dcells[loc[k]].emplace_back((int32_t)c, k);
                    pos[loc[k]] = dof_pos(c, k);
                }
            }
            for (int a = 0; a < dpc; ++a)
                if (loc[a] >= 0)
                    for (int b = 0; b < dpc; ++b)
                        if (loc[b] >= 0) adj[loc[a]].push_back(loc[b]);
        }
        for (auto& v : adj) {
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
        }
        // Order-2 cell bubbles are condensed cell by cell and ordered last;
        // the block-tridiagonal levels cover the edge DOFs only.
        std::vector<uint8_t> bub(n, 0);
        int64_t nbub = 0;
        if (m->order == 2)
            for (int64_t i = 0; i < n; ++i)
                if (gd[i] >= 2 * m->n_edge) { bub[i] = 1; ++nbub; }
        // BFS levels from the DOFs at the smallest sweep coordinate
        double pmin = 1e300, pmax = -1e300;
        for (int64_t i = 0; i < n; ++i)
            if (!bub[i]) { pmin = std::min(pmin, pos[i]); pmax = std::max(pmax, pos[i]); }
        double tol = 1e-9 * (pmax - pmin + 1.0);
        std::vector<int32_t> lev(n, -1);
        std::vector<int32_t> frontier;
        for (int64_t i = 0; i < n; ++i)
            if (!bub[i] && pos[i] <= pmin + tol) { lev[i] = 0; frontier.push_back((int32_t)i); }
        int nl = 1;
        auto bfs = [&](std::vector<int32_t>& fr) {
            while (!fr.empty()) {
                std::vector<int32_t> nxt;
                for (int32_t i : fr)
                    for (int32_t j : adj[i])
                        if (!bub[j] && lev[j] < 0) { lev[j] = nl; nxt.push_back(j); }
                if (!nxt.empty()) ++nl;
                fr.swap(nxt);
            }
        };
        bfs(frontier);
        for (int64_t i = 0; i < n; ++i)
            if (!bub[i] && lev[i] < 0) {       // disconnected piece: start a new BFS there
                std::vector<int32_t> fr{(int32_t)i};
                lev[i] = nl++;
                bfs(fr);
            }
        // merge consecutive BFS levels into blocks of <= max_block DOFs
        std::vector<int64_t> cnt(nl, 0);
        for (int64_t i = 0; i < n; ++i)
            if (!bub[i]) cnt[lev[i]]++;
        std::vector<int32_t> blk_of(nl);
        std::vector<int64_t> bsize;
        for (int l = 0; l < nl; ++l) {
            if (cnt[l] == 0) { blk_of[l] = bsize.empty() ? 0 : (int32_t)bsize.size() - 1; continue; }
            if (!bsize.empty() && bsize.back() + cnt[l] <= m->max_block) {
                bsize.back() += cnt[l];
            } else {
                bsize.push_back(cnt[l]);
            }
            blk_of[l] = (int32_t)bsize.size() - 1;
        }
        // local order: (block, global id) for edge DOFs, then bubbles by global id
        std::vector<int64_t> order(n);
        std::iota(order.begin(), order.end(), 0);
        auto key = [&](int64_t a) -> int64_t { return bub[a] ? (int64_t)INT32_MAX : blk_of[lev[a]]; };
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key(a) < key(b); });
        std::vector<int32_t> newid(n);
        for (int64_t i = 0; i < n; ++i) newid[order[i]] = (int32_t)i;
        m->subs[s].off = off;
        m->subs[s].n = n;
        m->subs[s].ne = n - nbub;
        THM_REQUIRE(nbub % 4 == 0, "internal: order-2 bubbles not in groups of 4");
        m->subs[s].cell0 = (int32_t)m->n_bcell;
        m->n_bcell += nbub / 4;
        m->subs[s].lev0 = (int32_t)m->levels.size();
        m->subs[s].nlev = (int32_t)bsize.size();
        int32_t st = (int32_t)off;
        for (size_t b = 0; b < bsize.size(); ++b) {
            Level L{};
            L.start = st;
            L.size = (int32_t)bsize[b];
            st += L.size;
            m->levels.push_back(L);
        }
        for (int64_t i = 0; i < n; ++i) {
            int64_t o = order[i];
            m->loc_gdof.push_back(gd[o]);
            m->loc_sub.push_back(s);
            std::vector<int32_t> cols;
            for (int32_t j : adj[o]) cols.push_back((int32_t)(off + newid[j]));
            std::sort(cols.begin(), cols.end());
            row_cols_all.push_back(std::move(cols));
            auto dc = dcells[o];
            std::sort(dc.begin(), dc.end());
            THM_REQUIRE((int)dc.size() <= m->maxc, "internal: too many cells per DOF");
            for (int t = 0; t < m->maxc; ++t) {
                row_cell_v.push_back(t < (int)dc.size() ? dc[t].first : -1);
                row_k_v.push_back(t < (int)dc.size() ? dc[t].second : -1);
            }
        }
        for (int64_t c : cs)
            for (int k = 0; k < dpc; ++k) {
                int64_t g = m->cell_dofs[c * dpc + k];
                m->cell_loc[c * dpc + k] = m->is_dir[g] ? -1 : (int32_t)(off + newid[lid(g)]);
            }
        off += n;
    }
    m->n_loc = off;
    m->row_cell.swap(row_cell_v);
    m->row_k.swap(row_k_v);

    // ---- level offsets into the factor storage (rows padded to a multiple
    //      of 4 entries, so every row and every block is 16-byte aligned) and
    //      the middle level of the twisted factorisation: the level that
    //      balances the factor bytes (plus a per-level latency allowance) of
    //      the two chains
    m->max_m = 0;
    m->max_lev = 0;
    m->bt_nvec = 0;
    int64_t fo = 0;
    for (int s = 0; s < ns; ++s) {
        auto& S = m->subs[s];
        m->max_lev = std::max(m->max_lev, S.nlev);
        std::vector<double> cost(S.nlev);
        for (int l = 0; l < S.nlev; ++l) {
            Level& L = m->levels[S.lev0 + l];
            L.prev = l > 0 ? m->levels[S.lev0 + l - 1].size : 0;
            L.next = l + 1 < S.nlev ? m->levels[S.lev0 + l + 1].size : 0;
            m->max_m = std::max(m->max_m, L.size);
            L.offW = fo;
            fo += (int64_t)L.size * (((int64_t)L.size + 3) / 4 * 4);
            cost[l] = (double)L.size * L.size + 16384.0;
        }
        S.kmid = 0;
        if (S.nlev > 0) {
            double tot = 0, below = 0, best = 1e300;
            for (double c : cost) tot += c;
            for (int k = 0; k < S.nlev; ++k) {
                const double above = tot - below - cost[k];
                const double w = std::max(below, above);
                if (w < best) { best = w; S.kmid = k; }
                below += cost[k];
            }
            const Level& Lk = m->levels[S.lev0 + S.kmid];
            const Level& L0 = m->levels[S.lev0];
            const Level& Le = m->levels[S.lev0 + S.nlev - 1];
            m->bt_nvec = std::max<int64_t>(m->bt_nvec, (int64_t)Lk.start + Lk.size - L0.start);
            m->bt_nvec = std::max<int64_t>(m->bt_nvec, (int64_t)Le.start + Le.size - Lk.start);
        }
    }
    // H_l^T after all W blocks: rows of the level the backward sweep comes
    // from (l + 1 above the middle, l - 1 below it), stride r4(m_l)
    for (int s = 0; s < ns; ++s) {
        const auto& S = m->subs[s];
        for (int l = 0; l < S.nlev; ++l) {
            Level& L = m->levels[S.lev0 + l];
            if (l == S.kmid) {
                L.offH = -1;
                continue;
            }
            const int nb = l < S.kmid ? L.next : L.prev;
            L.offH = fo;
            fo += (int64_t)nb * (((int64_t)L.size + 3) / 4 * 4);
        }
    }
    m->fac_elems = fo + 4;

    // ---- SELL-32 pattern
    m->n_slices = (m->n_loc + SELL_C - 1) / SELL_C;
    m->slice_ptr.assign(m->n_slices + 1, 0);
    for (int64_t sl = 0; sl < m->n_slices; ++sl) {
        size_t w = 0;
        for (int64_t r = sl * SELL_C; r < std::min<int64_t>(m->n_loc, (sl + 1) * SELL_C); ++r)
            w = std::max(w, row_cols_all[r].size());
        m->slice_ptr[sl + 1] = m->slice_ptr[sl] + (int64_t)w * SELL_C;
    }
    m->n_slots = m->slice_ptr[m->n_slices];
    m->sell_col.assign(m->n_slots, 0);
    m->sell_pad.assign(m->n_slots, 1);
    for (int64_t sl = 0; sl < m->n_slices; ++sl) {
        int64_t w = (m->slice_ptr[sl + 1] - m->slice_ptr[sl]) / SELL_C;
        for (int lane = 0; lane < SELL_C; ++lane) {
            int64_t r = sl * SELL_C + lane;
            for (int64_t t = 0; t < w; ++t) {
                int64_t idx = m->slice_ptr[sl] + t * SELL_C + lane;
                if (r < m->n_loc && t < (int64_t)row_cols_all[r].size()) {
                    m->sell_col[idx] = row_cols_all[r][t];
                    m->sell_pad[idx] = 0;
                } else {
                    m->sell_col[idx] = (int32_t)std::min<int64_t>(r, m->n_loc - 1);
                }
            }
        }
    }
    m->col16 = true;
    for (const auto& S : m->subs) m->col16 = m->col16 && S.n <= 65536;
    if (m->col16) {
        m->sell_col16.assign(m->n_slots, 0);
        for (int64_t sl = 0; sl < m->n_slices; ++sl) {
            int64_t w = (m->slice_ptr[sl + 1] - m->slice_ptr[sl]) / SELL_C;
            for (int lane = 0; lane < SELL_C; ++lane) {
                int64_t r = sl * SELL_C + lane;
                if (r >= m->n_loc) continue;                  // never read (beyond the last row)
                const int64_t off = m->subs[m->loc_sub[r]].off;
                for (int64_t t = 0; t < w; ++t) {
                    const int64_t idx = m->slice_ptr[sl] + t * SELL_C + lane;
                    const int64_t rel = m->sell_col[idx] - off;
                    THM_REQUIRE(rel >= 0 && rel < 65536, "SpMV column outside its row's subdomain");
                    m->sell_col16[idx] = (uint16_t)rel;
                }
            }
        }
    }
    // ---- level coupling lists: for every level row, its S entries in the
    //      previous level (E_l) and in the next level (F_l), one 16-byte
    //      aligned block per (level, side)
    m->cpl_ptr.clear(); m->cpl_col.clear(); m->cpl_slot.clear();
    m->max_cnz = 0;
    m->max_ne = 0;
    auto pad4i = [](std::vector<int32_t>& v) { while (v.size() % 4) v.push_back(0); };
    for (int s = 0; s < ns; ++s) {
        const auto& S = m->subs[s];
        m->max_ne = std::max<int64_t>(m->max_ne, S.ne);
        for (int l = 0; l < S.nlev; ++l) {
            Level& L = m->levels[S.lev0 + l];
            for (int side = 0; side < 2; ++side) {
                int64_t c0 = side == 0 ? (int64_t)L.start - L.prev : (int64_t)L.start + L.size;
                int64_t c1 = side == 0 ? (int64_t)L.start : c0 + L.next;
                pad4i(m->cpl_ptr);
                while (m->cpl_col.size() % 4) { m->cpl_col.push_back(0); m->cpl_slot.push_back(-1); }
                int64_t p0 = (int64_t)m->cpl_ptr.size(), q0 = (int64_t)m->cpl_col.size();
                for (int i = 0; i <= L.size; ++i) {
                    m->cpl_ptr.push_back((int32_t)(m->cpl_col.size() - q0));
                    if (i == L.size) break;
                    int64_t r = L.start + i;
                    int64_t sl = r / SELL_C;
                    int lane = (int)(r % SELL_C);
                    int64_t w = (m->slice_ptr[sl + 1] - m->slice_ptr[sl]) / SELL_C;
                    for (int64_t t = 0; t < w; ++t) {
                        int64_t idx = m->slice_ptr[sl] + t * SELL_C + lane;
                        if (m->sell_pad[idx]) continue;
                        int64_t c = m->sell_col[idx];
                        if (c >= c0 && c < c1) {
                            m->cpl_col.push_back((int32_t)(c - c0));
                            m->cpl_slot.push_back(idx);
                        }
                    }
                }
                int32_t nz = (int32_t)(m->cpl_col.size() - q0);
                m->max_cnz = std::max(m->max_cnz, nz);
                if (side == 0) { L.eptr = p0; L.eoff = q0; L.enz = nz; }
                else { L.fptr = p0; L.foff = q0; L.fnz = nz; }
            }
        }
    }
    pad4i(m->cpl_ptr);
    for (int k = 0; k < 8; ++k) { m->cpl_ptr.push_back(0); m->cpl_col.push_back(0); m->cpl_slot.push_back(-1); }
    // values one block solve reads per subdomain (the byte model of the
    // block-solve kernel): the factor blocks and coupling lists it streams,
    // and the order-2 condensation tables
    m->bt_welem.assign(ns, 0);
    for (int s = 0; s < ns; ++s) {
        const auto& S = m->subs[s];
        int64_t w = bt_stream_values(S, m->levels.data());
        if (m->order == 2) w += 8 * S.ne + 12 * (S.n - S.ne);
        m->bt_welem[s] = w;
    }
    THM_REQUIRE(m->cpl_col.size() < (size_t)INT32_MAX, "coupling lists too large");
    row_cols_all.clear();

    // ---- reduction chunks
    m->chunks.clear();
    for (int s = 0; s < ns; ++s) {
        const auto& S = m->subs[s];
        for (int64_t b = 0; b < S.n; b += CHUNK) {
            Chunk ch{};
            ch.seg = s;
            ch.begin = S.off + b;
            ch.end = S.off + std::min<int64_t>(S.n, b + CHUNK);
            m->chunks.push_back(ch);
        }
    }

    // ---- global <-> local maps
    m->owner_loc.assign(m->n_dof, -1);
    std::vector<int64_t> ccount(m->n_dof + 1, 0);
    for (int64_t r = 0; r < m->n_loc; ++r) ccount[m->loc_gdof[r] + 1]++;
    m->copy_ptr.assign(m->n_dof + 1, 0);
    for (int64_t g = 0; g < m->n_dof; ++g) m->copy_ptr[g + 1] = m->copy_ptr[g] + ccount[g + 1];
    m->copy_idx.assign(m->n_loc, 0);
    std::vector<int64_t> fill(m->copy_ptr.begin(), m->copy_ptr.end() - 1);
    for (int64_t r = 0; r < m->n_loc; ++r) m->copy_idx[fill[m->loc_gdof[r]]++] = (int32_t)r;  // ascending subdomain
    m->loc_is_owner.assign(m->n_loc, 0);
    for (int64_t g = 0; g < m->n_dof; ++g)
        if (m->copy_ptr[g + 1] > m->copy_ptr[g]) {
            m->owner_loc[g] = m->copy_idx[m->copy_ptr[g]];
            m->loc_is_owner[m->owner_loc[g]] = 1;
        } else {
            THM_REQUIRE(m->is_dir[g], "internal: free DOF without a subdomain copy");
        }

    // ---- faces with impedance (Gamma^inf, kind 1) or transmission (Sigma, kind 2)
    //      terms: 2-D faces are edges (1 or 2 DOFs), 3-D faces are quads (4
    //      edge DOFs); the tangential face mass couples the face's DOFs
    constexpr int RF = thm_mesh::RF;
    m->fd = d == 2 ? (m->order == 1 ? 1 : 2) : 4;
    const int fd = m->fd;
    m->face_v.clear(); m->face_dof.clear(); m->face_sgn.clear(); m->face_kind.clear(); m->face_sub.clear();
    auto add_face = [&](const int64_t* fv, int kind, int s0, int s1) {
        int32_t v[4] = {(int32_t)fv[0], (int32_t)fv[1], d == 3 ? (int32_t)fv[2] : 0, d == 3 ? (int32_t)fv[3] : 0};
        for (int k = 0; k < 4; ++k) m->face_v.push_back(v[k]);
        if (d == 2) {
            int64_t e = host_find_edge(m, fv[0], fv[1]);
            int8_t sg = fv[0] < fv[1] ? 1 : -1;
            if (m->order == 1) { m->face_dof.push_back((int32_t)e); m->face_sgn.push_back(sg); }
            else {
                m->face_dof.push_back((int32_t)(2 * e)); m->face_sgn.push_back(sg);
                m->face_dof.push_back((int32_t)(2 * e + 1)); m->face_sgn.push_back(1);
            }
        } else {
            for (int k = 0; k < 4; ++k) {
                int64_t a = fv[h_edges2[k][0]], b = fv[h_edges2[k][1]];
                m->face_dof.push_back((int32_t)host_find_edge(m, a, b));
                m->face_sgn.push_back(a < b ? 1 : -1);
            }
        }
        m->face_kind.push_back((int8_t)kind);
        m->face_sub.push_back(s0);
        m->face_sub.push_back(s1);
    };
    if (d == 2) {
        for (int64_t e = 0; e < m->n_edge; ++e) {
            int32_t c0 = ecell[2 * e], c1 = ecell[2 * e + 1];
            int64_t fv[2] = {m->edge_lo[e], m->edge_hi[e]};
            if (c1 < 0 && edge_kind[e] == 1) add_face(fv, 1, m->cell_sub[c0], -1);
            else if (c1 >= 0 && m->cell_sub[c0] != m->cell_sub[c1]) add_face(fv, 2, m->cell_sub[c0], m->cell_sub[c1]);
        }
    } else {
        // all hex faces keyed by their sorted vertices
        struct FK { int64_t k[4]; int32_t cell; int8_t lf; };
        std::vector<FK> fk;
        fk.reserve(m->n_cell * 6);
        static const int lfaces[6][4] = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
        for (int64_t c = 0; c < m->n_cell; ++c)
            for (int f = 0; f < 6; ++f) {
                FK x;
                for (int k = 0; k < 4; ++k) x.k[k] = m->cells[c * 8 + lfaces[f][k]];
                std::sort(x.k, x.k + 4);
                x.cell = (int32_t)c; x.lf = (int8_t)f;
                fk.push_back(x);
            }
        auto less = [](const FK& a, const FK& b) {
            for (int k = 0; k < 4; ++k)
                if (a.k[k] != b.k[k]) return a.k[k] < b.k[k];
            return a.cell < b.cell;
        };
        std::sort(fk.begin(), fk.end(), less);
        auto same = [](const FK& a, const FK& b) { return std::equal(a.k, a.k + 4, b.k); };
        // impedance boundary faces: sorted keys of tag-0 bfaces
        std::vector<std::array<int64_t, 4>> imp;
        for (int64_t f = 0; f < m->n_bface; ++f)
            if (m->btag[f] == THM_TAG_IMPEDANCE) {
                std::array<int64_t, 4> k{m->bfaces[f * 4], m->bfaces[f * 4 + 1], m->bfaces[f * 4 + 2], m->bfaces[f * 4 + 3]};
                std::sort(k.begin(), k.end());
                imp.push_back(k);
            }
        std::sort(imp.begin(), imp.end());
        for (size_t p = 0; p < fk.size();) {
            size_t q = p + 1;
            while (q < fk.size() && same(fk[p], fk[q])) ++q;
            THM_REQUIRE(q - p <= 2, "a face is shared by more than two cells");
            int64_t fv[4];
            for (int k = 0; k < 4; ++k) fv[k] = m->cells[(int64_t)fk[p].cell * 8 + lfaces[fk[p].lf][k]];
            if (q - p == 1) {
                std::array<int64_t, 4> k{fk[p].k[0], fk[p].k[1], fk[p].k[2], fk[p].k[3]};
                if (std::binary_search(imp.begin(), imp.end(), k)) add_face(fv, 1, m->cell_sub[fk[p].cell], -1);
            } else if (m->cell_sub[fk[p].cell] != m->cell_sub[fk[p + 1].cell]) {
                add_face(fv, 2, m->cell_sub[fk[p].cell], m->cell_sub[fk[p + 1].cell]);
            }
            p = q;
        }
    }
    m->n_face = (int64_t)m->face_kind.size();
    auto loc_in = [&](int64_t g, int s) -> int32_t {
        if (s < 0 || m->is_dir[g]) return -1;
        for (int64_t p = m->copy_ptr[g]; p < m->copy_ptr[g + 1]; ++p)
            if (m->loc_sub[m->copy_idx[p]] == s) return m->copy_idx[p];
        return -1;
    };
    m->face_loc.assign(m->n_face * 2 * fd, -1);
    for (int64_t f = 0; f < m->n_face; ++f)
        for (int side = 0; side < 2; ++side)
            for (int a = 0; a < fd; ++a)
                m->face_loc[(f * 2 + side) * fd + a] = loc_in(m->face_dof[f * fd + a], m->face_sub[f * 2 + side]);
    // per local row: the faces (of its subdomain) whose terms reach it
    m->row_face.assign(m->n_loc * RF, -1);
    m->row_face_a.assign(m->n_loc * RF, 0);
    m->row_face_side.assign(m->n_loc * RF, 0);
    {
        std::vector<int> cnt(m->n_loc, 0);
        for (int64_t f = 0; f < m->n_face; ++f)
            for (int side = 0; side < 2; ++side)
                for (int a = 0; a < fd; ++a) {
                    int32_t r = m->face_loc[(f * 2 + side) * fd + a];
                    if (r < 0) continue;
                    THM_REQUIRE(cnt[r] < RF, "internal: too many boundary faces at one DOF");
                    m->row_face[r * RF + cnt[r]] = (int32_t)f;
                    m->row_face_a[r * RF + cnt[r]] = (int8_t)a;
                    m->row_face_side[r * RF + cnt[r]] = (int8_t)side;
                    cnt[r]++;
                }
    }
    // interface entries: one per (receiver i, sender j, free DOF g on Sigma_ij),
    // with the terms (face, a, b, sender column) of (M_Sigma_ij u_j)[g]
    struct Term { int32_t i, j; int64_t g; int32_t f; int8_t a, b; int32_t col; };
    std::vector<Term> terms;
    for (int64_t f = 0; f < m->n_face; ++f) {
        if (m->face_kind[f] != 2) continue;
        for (int side = 0; side < 2; ++side) {
            const int i = m->face_sub[f * 2 + side], j = m->face_sub[f * 2 + 1 - side];
            for (int a = 0; a < fd; ++a) {
                if (m->face_loc[(f * 2 + side) * fd + a] < 0) continue;       // Dirichlet DOF: no entry
                const int64_t g = m->face_dof[f * fd + a];
                for (int b = 0; b < fd; ++b) {
                    int32_t col = m->face_loc[(f * 2 + 1 - side) * fd + b];
                    if (col < 0) col = -(m->face_dof[f * fd + b] + 1);
                    terms.push_back({i, j, g, (int32_t)f, (int8_t)a, (int8_t)b, col});
                }
            }
        }
    }
    std::sort(terms.begin(), terms.end(), [](const Term& x, const Term& y) {
        if (x.i != y.i) return x.i < y.i;
        if (x.j != y.j) return x.j < y.j;
        if (x.g != y.g) return x.g < y.g;
        if (x.f != y.f) return x.f < y.f;
        return x.b < y.b;
    });
    m->if_recv.clear(); m->if_send.clear(); m->if_gdof.clear(); m->if_rowi.clear();
    m->if_ptr.assign(1, 0); m->if_tf.clear(); m->if_ta.clear(); m->if_tb.clear(); m->if_tcol.clear();
    for (size_t p = 0; p < terms.size(); ++p) {
        const Term& t = terms[p];
        if (p == 0 || t.i != terms[p - 1].i || t.j != terms[p - 1].j || t.g != terms[p - 1].g) {
            if (p > 0) m->if_ptr.push_back((int64_t)m->if_tf.size());
            m->if_recv.push_back(t.i); m->if_send.push_back(t.j); m->if_gdof.push_back(t.g);
            m->if_rowi.push_back(loc_in(t.g, t.i));
            THM_REQUIRE(m->if_rowi.back() >= 0, "internal: interface DOF without a receiver copy");
        }
        m->if_tf.push_back(t.f); m->if_ta.push_back(t.a); m->if_tb.push_back(t.b); m->if_tcol.push_back(t.col);
    }
    if (!terms.empty()) m->if_ptr.push_back((int64_t)m->if_tf.size());
    m->n_if = (int64_t)m->if_recv.size();
    m->if_partner.assign(m->n_if, -1);
    for (int64_t k = 0; k < m->n_if; ++k) {
        // partner entry (j <- i, same DOF): binary search in the sorted entry list
        int64_t lo = 0, hi = m->n_if - 1, found = -1;
        const int32_t ki = m->if_send[k], kj = m->if_recv[k];
        const int64_t kg = m->if_gdof[k];
        while (lo <= hi) {
            int64_t mid = (lo + hi) / 2;
            auto c = std::make_tuple(m->if_recv[mid], m->if_send[mid], m->if_gdof[mid]);
            auto w = std::make_tuple(ki, kj, kg);
            if (c == w) { found = mid; break; }
            if (c < w) lo = mid + 1; else hi = mid - 1;
        }
        THM_REQUIRE(found >= 0, "internal: interface entry without partner");
        m->if_partner[k] = (int32_t)found;
    }
    m->rowg_ptr.assign(m->n_loc + 1, 0);
    for (int64_t k = 0; k < m->n_if; ++k) m->rowg_ptr[m->if_rowi[k] + 1]++;
    for (int64_t r = 0; r < m->n_loc; ++r) m->rowg_ptr[r + 1] += m->rowg_ptr[r];
    m->rowg_idx.assign(m->n_if, 0);
    {
        std::vector<int64_t> f2(m->rowg_ptr.begin(), m->rowg_ptr.end() - 1);
        for (int64_t k = 0; k < m->n_if; ++k) m->rowg_idx[f2[m->if_rowi[k]]++] = (int32_t)k;
    }

    // ---- device mirrors
    std::vector<int32_t> cl32(m->cell_loc.begin(), m->cell_loc.end());
    m->d_cell_loc.upload(cl32);
    m->d_sell_col.upload(m->sell_col);
    if (m->col16) m->d_sell_col16.upload(m->sell_col16);
    m->d_sell_pad.upload(m->sell_pad);
    m->d_slice_ptr.upload(m->slice_ptr);
    m->d_row_cell.upload(m->row_cell);
    m->d_row_k.upload(m->row_k);
    m->d_face_v.upload(m->face_v);
    m->d_face_dof.upload(m->face_dof);
    m->d_face_sgn.upload(m->face_sgn);
    m->d_face_kind.upload(m->face_kind);
    m->d_face_loc.upload(m->face_loc);
    m->d_row_face.upload(m->row_face);
    m->d_row_face_a.upload(m->row_face_a);
    m->d_row_face_side.upload(m->row_face_side);
    m->d_if_ptr.upload(m->if_ptr);
    m->d_if_tf.upload(m->if_tf);
    m->d_if_ta.upload(m->if_ta);
    m->d_if_tb.upload(m->if_tb);
    m->d_if_tcol.upload(m->if_tcol);
    m->d_levels.upload(m->levels);
    m->d_cpl_ptr.upload(m->cpl_ptr);
    m->d_cpl_col.upload(m->cpl_col);
    m->d_cpl_slot.upload(m->cpl_slot);
    m->d_subs.upload(m->subs);
    m->d_bt_welem.upload(m->bt_welem);
    m->d_chunks.upload(m->chunks);
    m->d_dir_edges.upload(m->dir_edges);
    m->dir_dofs.clear();
    for (int64_t g = 0; g < m->n_dof; ++g)
        if (m->is_dir[g]) m->dir_dofs.push_back(g);
    m->d_dir_dofs.upload(m->dir_dofs);
    m->d_loc_gdof.upload(m->loc_gdof);
    m->d_loc_sub.upload(m->loc_sub);
    m->d_if_rowi.upload(m->if_rowi);
    m->d_if_partner.upload(m->if_partner);
    m->d_rowg_ptr.upload(m->rowg_ptr);
    m->d_rowg_idx.upload(m->rowg_idx);
    m->d_owner_loc.upload(m->owner_loc);
    m->d_copy_ptr.upload(m->copy_ptr);
    m->d_copy_idx.upload(m->copy_idx);
    m->d_loc_is_owner.upload(m->loc_is_owner);
    m->loc_is_bub.assign(m->n_loc, 0);
    if (m->order == 2)
        for (int64_t r = 0; r < m->n_loc; ++r) m->loc_is_bub[r] = m->loc_gdof[r] >= 2 * m->n_edge;
    m->d_loc_is_bub.upload(m->loc_is_bub);
    THM_CUDA(cudaDeviceSynchronize());
}

}  // namespace thm

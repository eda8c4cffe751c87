// x = P_i^{-1} r for every subdomain at once (the block preconditioner of
// Eq. 7: the same real P_i^{-1} applied to the real and the imaginary part).
//
// P_i (for order 2 its edge Schur complement after the per-cell bubble
// condensation) is block tridiagonal over the BFS levels l = 0..L-1 of the
// subdomain's DOF graph, with diagonal blocks D_l and couplings
// E_l = P_{l,l-1}, F_l = P_{l,l+1} = E_{l+1}^T.  It is factored from both
// ends towards a middle level k (a "twisted" block LU):
//   top    (l < k):  S_0 = D_0,      S_l = D_l - E_l S_{l-1}^{-1} F_{l-1}
//   bottom (l > k):  S_{L-1} = D_{L-1}, S_l = D_l - F_l S_{l+1}^{-1} E_{l+1}
//   middle:          S_k = D_k - E_k S_{k-1}^{-1} F_{k-1} - F_k S_{k+1}^{-1} E_{k+1}
// and only the dense W_l = S_l^{-1} are stored (row stride r4(m_l), symmetric).
// The solve runs the two chains concurrently on the two CTAs of a cluster:
//   rank 0, l = 0..k-1:    z_l = W_l (r_l - E_l z_{l-1})
//   rank 1, l = L-1..k+1:  z_l = W_l (r_l - F_l z_{l+1})
//   middle, both ranks:    x_k = W_k (r_k - E_k z_{k-1} - F_k z_{k+1})
//                          (each rank forms its own coupling term and half of
//                           the product; the halves meet through DSMEM)
//   rank 0, l = k-1..0:    x_l = z_l - H_l x_{l+1},   H_l = W_l F_l
//   rank 1, l = k+1..L-1:  x_l = z_l - H_l x_{l-1},   H_l = W_l E_l
// so each SM streams half of the factor and the dependent chain is half as
// long as a one-sided sweep.  The dense H_l (stored transposed; the
// factorisation forms them in its Schur updates) make a backward step one
// GEMV with no sparse coupling phase, for as many bytes as W_l would stream.
//
// Per CTA, one producer warp streams the tiles (the coupling CSR block of a
// step, then row tiles of W_l) with 1-D TMA bulk copies into two rings of
// shared-memory slots (full/empty mbarriers): large slots for the W tiles,
// small ones for the coupling blocks, so that a few-KB coupling block does not
// hold a W-sized slot and the W ring reaches further ahead.  When a coupling
// block is too large for a small slot (3-D levels of several hundred rows),
// the consumers read it from global memory instead (cglob); a level step then
// streams megabytes of W, next to which those loads are cheap.  12 consumer warps hold the
// CTA's half of the subdomain vector in shared memory and run the block
// GEMVs, both vector components at once (each W element feeds two FMAs).
// Every wait is bounded: on expiry the CTA raises *err, stops issuing, lets
// its copies in flight land and finishes its (then meaningless) control flow
// so that no barrier is left waiting.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "kernels.cuh"

namespace thm {

constexpr int BT_NT = 384;                  // consumer threads
constexpr int BT_NW = BT_NT / 32;           // consumer warps
constexpr int BT_THREADS = BT_NT + 32;      // + one producer warp
// GEMV layout: a warp pass covers GQ = 8 output quads with 4 row subsets, and
// a warp holds at most GMAX quad groups, so m_l <= 4 * GQ * GMAX * BT_NW.  The
// 8 lanes of a quarter-warp read 128 contiguous bytes of one W row, so the
// loads are free of bank conflicts whatever the row stride.  Narrower groups
// keep more warps busy on 130-row levels but measured slower: 4 quads x 8 row
// subsets 2024 against 1687 cycles per 130 x 132 tile alone (two rows 16 B
// apart meet in the banks of one quarter-warp), 2 quads x 16 subsets 139
// against 116 us per launch.
constexpr int BT_GQ = 8;
constexpr int BT_GMAX = 4;
constexpr int BT_MAX_M = 4 * BT_GQ * BT_GMAX * BT_NW;     // 1536
constexpr int BT_NC = 4;                    // slots of the coupling ring
constexpr int BT_PROW_A = 4;                // rows per pass of the order-2 prologue (a)
constexpr int BT_PROW_C = 3;                // and of the epilogue (c)

__host__ __device__ constexpr int bt_r4(int v) { return (v + 3) / 4 * 4; }
__host__ __device__ constexpr size_t bt_r16(size_t v) { return (v + 15) / 16 * 16; }

// One step of a rank's chain: level l, coupling block (0 none, 1 E_l to
// level l-1, 2 F_l to level l+1), the rows [ra, rb) this rank streams (of W_l;
// of H_l^T on a backward step, whose rows belong to the level nb it comes
// from), and the kind (0 forward, 1 middle, 2 backward).
struct BtStep {
    int l, cpl, ra, rb, kind, nb;
};

__device__ __forceinline__ int bt_nsteps(int rank, int L, int k) { return 2 * (rank == 0 ? k : L - 1 - k) + 1; }

__device__ __forceinline__ BtStep bt_step(int rank, int L, int k, int i, const Level* lv) {
    BtStep s;
    const int nf = rank == 0 ? k : L - 1 - k;
    if (i < nf) {
        s.kind = 0;
        s.l = rank == 0 ? i : L - 1 - i;
        s.cpl = i == 0 ? 0 : (rank == 0 ? 1 : 2);
    } else if (i == nf) {
        s.kind = 1;
        s.l = k;
        s.cpl = nf == 0 ? 0 : (rank == 0 ? 1 : 2);
    } else {
        s.kind = 2;
        const int d = i - nf;
        s.l = rank == 0 ? k - d : k + d;
        s.cpl = 0;
    }
    s.nb = rank == 0 ? s.l + 1 : s.l - 1;        // the backward step's input level
    const int m = lv[s.l].size;
    if (s.kind == 1) {
        const int h = m / 2;
        s.ra = rank == 0 ? 0 : h;
        s.rb = rank == 0 ? h : m;
    } else {
        s.ra = 0;
        s.rb = s.kind == 2 ? lv[s.nb].size : m;
    }
    return s;
}

// ---- cluster-scope mbarrier helpers ---------------------------------------
__device__ __forceinline__ unsigned mapa_u32(const void* p, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(unsigned cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];\n" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_try_cluster(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete
// sleeps (up to the hint) instead of spinning, so waiting warps take no issue
// slots from the working ones.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(2000u)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_try_cluster_sleep(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(2000u)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long bt_now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait (limit_ns of wall time, 1 s by default) that gives up at once
// when the CTA has already aborted; on expiry it raises the abort flag and *err.
template <bool CLUSTER>
__device__ __forceinline__ bool bt_wait(uint64_t* bar, unsigned parity, volatile int* abort, int* err,
                                        unsigned long long limit_ns) {
    if (CLUSTER ? mbar_try_cluster(bar, parity) : mbar_try(bar, parity)) return true;
    const unsigned long long t0 = bt_now_ns();
    while (true) {
        if (CLUSTER ? mbar_try_cluster_sleep(bar, parity) : mbar_try_sleep(bar, parity)) return true;
        if (*abort) return false;
        if (bt_now_ns() - t0 > limit_ns) break;
    }
    *abort = 1;
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void bt_bar_consumers() { asm volatile("bar.sync 1, %0;\n" ::"n"(BT_NT) : "memory"); }

template <class F, class R>
__device__ __forceinline__ void bt_load4(const F* p, R* w);
template <>
__device__ __forceinline__ void bt_load4<float, float>(const float* p, float* w) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
template <>
__device__ __forceinline__ void bt_load4<float, double>(const float* p, double* w) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
template <>
__device__ __forceinline__ void bt_load4<double, double>(const double* p, double* w) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
}
template <>
__device__ __forceinline__ void bt_load4<double, float>(const double* p, float* w) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    w[0] = (float)a.x; w[1] = (float)a.y; w[2] = (float)b.x; w[3] = (float)b.y;
}

// Shared-memory layout of k_bt_solve (host and device agree through this).
struct BtLayout {
    size_t bars, lv, slots, cslots, vec, su, tx, rx, ry, total;
};
template <class V>
__host__ __device__ inline BtLayout bt_layout(int ns, int slot_bytes, int cslot_bytes, int max_lev, int nvec,
                                              int max_m) {
    BtLayout L;
    size_t o = 0;
    L.bars = o; o += bt_r16((size_t)(2 * ns + 2 * BT_NC + 2) * 8);
    L.lv = o; o += bt_r16((size_t)max_lev * sizeof(Level));
    L.slots = o; o += (size_t)ns * slot_bytes;
    L.cslots = o; o += (size_t)BT_NC * cslot_bytes;
    const size_t vm = bt_r16((size_t)bt_r4(max_m) * sizeof(V));
    L.vec = o; o += bt_r16((size_t)nvec * sizeof(V));
    L.su = o; o += vm;
    L.tx = o; o += vm;
    L.rx = o; o += vm;
    L.ry = o; o += vm;
    L.total = o;
    return L;
}

// W element types: real factors (Eq. 7) or complex ones (the full 2x2 block
// operator of Section 3.2, T_i^{-1}).
template <class T> struct BtCplx { static constexpr bool value = false; };
template <> struct BtCplx<float2> { static constexpr bool value = true; };
template <> struct BtCplx<double2> { static constexpr bool value = true; };

// acc[c] += W[j][4q + c] * s for one quad of one W row (real or complex W)
template <class FW, class Rt, class V>
__device__ __forceinline__ void bt_quad_fma(const FW* p, const V s, Rt (&acc)[4][2]) {
    if constexpr (BtCplx<FW>::value) {
        Rt wr[4], wi[4];
        if constexpr (sizeof(FW) == 8) {
            const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
            wr[0] = a.x; wi[0] = a.y; wr[1] = a.z; wi[1] = a.w; wr[2] = b.x; wi[2] = b.y; wr[3] = b.z; wi[3] = b.w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double2 v = reinterpret_cast<const double2*>(p)[c];
                wr[c] = (Rt)v.x;
                wi[c] = (Rt)v.y;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc[c][0] += wr[c] * s.x - wi[c] * s.y;
            acc[c][1] += wr[c] * s.y + wi[c] * s.x;
        }
    } else {
        Rt w[4];
        bt_load4<FW, Rt>(p, w);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc[c][0] += w[c] * s.x;
            acc[c][1] += w[c] * s.y;
        }
    }
}

// shared-memory loads by 32-bit shared-window address
__device__ __forceinline__ float4 bt_lds128(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ float2 bt_lds64(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
// acc[c] += w[c] * s for the four entries of one W quad (FP32)
__device__ __forceinline__ void bt_fma4(const float4 w, const float2 sv, float (&acc)[4][2]) {
    acc[0][0] = fmaf(w.x, sv.x, acc[0][0]); acc[0][1] = fmaf(w.x, sv.y, acc[0][1]);
    acc[1][0] = fmaf(w.y, sv.x, acc[1][0]); acc[1][1] = fmaf(w.y, sv.y, acc[1][1]);
    acc[2][0] = fmaf(w.z, sv.x, acc[2][0]); acc[2][1] = fmaf(w.z, sv.y, acc[2][1]);
    acc[3][0] = fmaf(w.w, sv.x, acc[3][0]); acc[3][1] = fmaf(w.w, sv.y, acc[3][1]);
}

// (b2)+(b3) of a level step: y = W_l^T s over the rows [ra, rb) of W_l that
// this rank streams, then the step's output (forward: z_l, middle: this
// rank's half of x_k, backward: x_l = z_l - y).  Warp w owns the quad groups
// g = w, w + NW, ... (GQ output quads each, at most GMAX per warp); inside a
// warp, lane = (row subset rs, quad qq): the GQ lanes of a subset read
// 16 * GQ contiguous bytes of one W row and the NRS = 32 / GQ subsets take
// every NRS-th row.  The subsets are summed with shuffles, so each output is
// complete inside one warp: no cross-warp combine.  Every W tile of the step
// is waited for and released by every consumer warp, whatever its share.
template <int GQ, int GMAX, class V, class FW>
__device__ __forceinline__ void bt_gemv(const BtStep& st, int m, int o, int ldm, int R, int ns, int slot_bytes,
                                        const unsigned char* slots, uint64_t* full, uint64_t* empty, int& t,
                                        const V* su, V* vec, V* tx, V* pry, int warp, int lane, volatile int* abort,
                                        int* err, unsigned long long wait_ns) {
    using Rt = typename VT<V>::R;
    constexpr int NRS = 32 / GQ;
    const int nq = ldm / 4;
    const int ngr = (nq + GQ - 1) / GQ;
    const int rs = lane / GQ, qq = lane % GQ;
    Rt acc[GMAX][4][2];
#pragma unroll
    for (int u = 0; u < GMAX; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[u][c][0] = acc[u][c][1] = 0;
    for (int r0 = st.ra; r0 < st.rb; r0 += R) {
        const int q = t % ns;
        bt_wait<false>(&full[q], (unsigned)((t / ns) & 1), abort, err, wait_ns);
        const FW* Wt = reinterpret_cast<const FW*>(slots + (size_t)q * slot_bytes);
        const int nr = min(R, st.rb - r0);
#pragma unroll
        for (int u = 0; u < GMAX; ++u) {
            const int quad = (warp + u * BT_NW) * GQ + qq;
            if (warp + u * BT_NW < ngr && quad < nq) {
                if constexpr (std::is_same<FW, float>::value && std::is_same<V, float2>::value) {
                    // real FP32 factors: 32-bit shared addresses stepped by
                    // the row stride, ROWS rows per pass (their loads in flight together)
                    constexpr int ROWS = 4;
                    const uint32_t wstep = (uint32_t)NRS * 4u * (uint32_t)ldm, sstep = (uint32_t)NRS * 8u;
                    uint32_t wa = smem_u32(Wt) + 16u * (uint32_t)quad + (uint32_t)rs * 4u * (uint32_t)ldm;
                    uint32_t sa = smem_u32(su + r0) + (uint32_t)rs * 8u;
                    int jj = rs;
                    for (; jj + (ROWS - 1) * NRS < nr; jj += ROWS * NRS) {
                        float4 wv[ROWS];
                        float2 sv[ROWS];
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) {
                            sv[r] = bt_lds64(sa + (uint32_t)r * sstep);
                            wv[r] = bt_lds128(wa + (uint32_t)r * wstep);
                        }
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) bt_fma4(wv[r], sv[r], acc[u]);
                        wa += (uint32_t)ROWS * wstep;
                        sa += (uint32_t)ROWS * sstep;
                    }
                    for (; jj < nr; jj += NRS, wa += wstep, sa += sstep) bt_fma4(bt_lds128(wa), bt_lds64(sa), acc[u]);
                } else {
                    const FW* wc = Wt + 4 * quad;
                    int jj = rs;
                    // four rows per pass: their loads are independent
                    for (; jj + 3 * NRS < nr; jj += 4 * NRS) {
                        V sj[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) sj[r] = su[r0 + jj + NRS * r];
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            bt_quad_fma<FW, Rt, V>(wc + (size_t)(jj + NRS * r) * ldm, sj[r], acc[u]);
                    }
                    for (; jj < nr; jj += NRS) bt_quad_fma<FW, Rt, V>(wc + (size_t)jj * ldm, su[r0 + jj], acc[u]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_local(&empty[q]);
        ++t;
    }
    // sum the row subsets by recursive halving over the lanes qq + GQ * rs of
    // a quad: each of the log2(NRS) shuffle rounds halves the values a lane
    // carries (6 shuffles per group instead of 16), and lane (rs, qq) ends
    // with values 2 rs and 2 rs + 1 of its quad, value 2c + z being
    // component z of output 4 quad + c: both components of output rs
    static_assert(GQ == 8, "the halving leaves two values (one output) per lane");
#pragma unroll
    for (int u = 0; u < GMAX; ++u) {
        if (warp + u * BT_NW >= ngr) break;              // uniform across the warp
        Rt a[8];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            a[2 * c] = acc[u][c][0];
            a[2 * c + 1] = acc[u][c][1];
        }
        int n = 8;
#pragma unroll
        for (int off = 16; off >= GQ; off >>= 1, n >>= 1) {
            const bool up = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (i < n / 2) {
                    const Rt send = up ? a[i] : a[i + n / 2];
                    const Rt keep = up ? a[i + n / 2] : a[i];
                    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
        }
        const int quad = (warp + u * BT_NW) * GQ + qq;
        if (quad < nq) {
            const int i = 4 * quad + rs;                     // both components of output rs of the quad
            if (i < m) {
                const V yv = mk<V>(a[0], a[1]);
                if (st.kind == 0) {
                    vec[o + i] = yv;
                } else if (st.kind == 1) {
                    tx[i] = yv;
                    pry[i] = yv;
                } else {
                    const V z = vec[o + i];
                    vec[o + i] = mk<V>(z.x - yv.x, z.y - yv.y);
                }
            }
        }
    }
}

// 416 threads = 13 warps, allocated as 16 (4 per SM sub-partition): at most
// 128 registers per thread (152 fails to launch)
template <class V, class F, class FW = F>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(BT_THREADS, 1)
k_bt_solve(const Sub* __restrict__ subs, const Level* __restrict__ levels, const FW* __restrict__ fac,
           const int32_t* __restrict__ cptr, const int32_t* __restrict__ ccol, const F* __restrict__ cval,
           int64_t n_loc, int condensed, const int32_t* __restrict__ ab, const F* __restrict__ av,
           const F* __restrict__ cv, const int32_t* __restrict__ e8, const F* __restrict__ ev, int R, int ns, int slot_bytes, int cslot_bytes, int cglob, int max_lev, int nvec,
           int max_m, unsigned long long wait_ns, int stall_w,
           int* __restrict__ err, const int* __restrict__ act, const int64_t* __restrict__ welem,
           unsigned long long* __restrict__ work, const V* __restrict__ x, V* __restrict__ y) {
    using Rt = typename VT<V>::R;
    namespace cg = cooperative_groups;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int peer = rank ^ 1;
    const BtLayout lay = bt_layout<V>(ns, slot_bytes, cslot_bytes, max_lev, nvec, max_m);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.bars);   // W ring
    uint64_t* empty = full + ns;
    uint64_t* cfull = empty + ns;                                      // coupling ring
    uint64_t* cempty = cfull + BT_NC;
    uint64_t* xbar = cempty + BT_NC;      // [0]: coupling terms of the middle level, [1]: halves of x_k
    Level* lv = reinterpret_cast<Level*>(smem + lay.lv);
    unsigned char* slots = smem + lay.slots;
    unsigned char* cslots = smem + lay.cslots;
    V* vec = reinterpret_cast<V*>(smem + lay.vec);
    V* su = reinterpret_cast<V*>(smem + lay.su);
    V* tx = reinterpret_cast<V*>(smem + lay.tx);
    V* rx = reinterpret_cast<V*>(smem + lay.rx);
    V* ry = reinterpret_cast<V*>(smem + lay.ry);
    V* prx = cluster.map_shared_rank(rx, peer);
    V* pry = cluster.map_shared_rank(ry, peer);
    volatile int* abort = &s_abort;

    // a subdomain whose Krylov segment has converged is skipped by both CTAs
    // of its cluster (same flag, read before any cluster barrier)
    if (act && !act[blockIdx.y]) return;
    const Sub S = subs[blockIdx.y];
    const int L = S.nlev, k = S.kmid;
    if (work && rank == 0 && threadIdx.x == 0) {       // instrumentation: the work this launch does
        atomicAdd(&work[0], (unsigned long long)welem[blockIdx.y]);
        atomicAdd(&work[1], (unsigned long long)S.n);
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int l = tid; l < L; l += blockDim.x) lv[l] = levels[S.lev0 + l];
    if (tid == 0) {
        s_abort = 0;
        for (int q = 0; q < ns; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], BT_NW);
        }
        for (int q = 0; q < BT_NC; ++q) {
            mbar_init(&cfull[q], 1);
            mbar_init(&cempty[q], BT_NW);
        }
        mbar_init(&xbar[0], BT_NW);
        mbar_init(&xbar[1], BT_NW);
        mbar_fence_init();
    }
    __syncthreads();
    cluster.sync();                       // the peer's barriers exist before any remote arrive

    const int nst = L > 0 ? bt_nsteps(rank, L, k) : 0;
    if (warp == BT_NW) {
        // ---------------- producer warp: lane 0 streams the tiles ----------------
        if (lane == 0 && nst > 0) {
            int pw = 0, pc = 0;                  // tiles issued into the W ring / the coupling ring
            bool ok = true;
            for (int si = 0; si < nst && ok; ++si) {
                const BtStep st = bt_step(rank, L, k, si, lv);
                const Level& Lv = lv[st.l];
                const int m = Lv.size, ldm = bt_r4(m);
                if (st.cpl && !cglob) {
                    const int q = pc % BT_NC, n = pc / BT_NC;
                    if (n > 0 && !bt_wait<false>(&cempty[q], (unsigned)((n - 1) & 1), abort, err, wait_ns)) { ok = false; break; }
                    unsigned char* dst = cslots + (size_t)q * cslot_bytes;
                    fence_proxy_async();
                    const bool e = st.cpl == 1;
                    const int64_t po = e ? Lv.eptr : Lv.fptr, qo = e ? Lv.eoff : Lv.foff;
                    const int nz = e ? Lv.enz : Lv.fnz;
                    const unsigned pb = (unsigned)bt_r16((size_t)(m + 1) * 4);
                    const unsigned cb = (unsigned)bt_r16((size_t)nz * 4);
                    const unsigned vb = (unsigned)bt_r16((size_t)nz * sizeof(F));
                    mbar_expect_tx(&cfull[q], pb + cb + vb);
                    tma_load_1d(dst, cptr + po, pb, &cfull[q]);
                    if (cb) tma_load_1d(dst + pb, ccol + qo, cb, &cfull[q]);
                    if (vb) tma_load_1d(dst + pb + cb, cval + qo, vb, &cfull[q]);
                    ++pc;
                }
                for (int r0 = st.ra; r0 < st.rb && ok; r0 += R, ++pw) {
                    const int q = pw % ns, n = pw / ns;
                    if (n > 0 && !bt_wait<false>(&empty[q], (unsigned)((n - 1) & 1), abort, err, wait_ns)) { ok = false; break; }
                    unsigned char* dst = slots + (size_t)q * slot_bytes;
                    fence_proxy_async();
                    const int nr = min(R, st.rb - r0);
                    const unsigned wb = (unsigned)((size_t)nr * ldm * sizeof(FW));
                    if (stall_w) continue;           // failure-detection test: the W tiles never come
                    mbar_expect_tx(&full[q], wb);
                    tma_load_1d(dst, fac + (st.kind == 2 ? Lv.offH : Lv.offW) + (int64_t)r0 * ldm, wb, &full[q]);
                }
            }
            // let every issued copy land before the CTA may leave
            for (int q = 0; q < ns && q < pw && !stall_w; ++q) {
                const int last = q + ((pw - 1 - q) / ns) * ns;      // last tile issued into slot q
                for (int it = 0; it < (1 << 22); ++it)
                    if (mbar_try(&full[q], (unsigned)((last / ns) & 1))) break;
            }
            for (int q = 0; q < BT_NC && q < pc; ++q) {
                const int last = q + ((pc - 1 - q) / BT_NC) * BT_NC;
                for (int it = 0; it < (1 << 22); ++it)
                    if (mbar_try(&cfull[q], (unsigned)((last / BT_NC) & 1))) break;
            }
        }
        __syncwarp();
    } else if (nst > 0) {
        // ---------------- consumer warps ----------------
        const int vbase = rank == 0 ? lv[0].start : lv[k].start;
        const int vend = rank == 0 ? lv[k].start + lv[k].size : lv[L - 1].start + lv[L - 1].size;
        // (a) load r for this rank's levels; order 2: r_E <- r_E - G r_I.
        // BT_PROW_A rows per pass: their table loads, then their gathers, are in
        // flight together (each row's arithmetic is unchanged).
        for (int e0 = vbase + tid; e0 < vend; e0 += BT_PROW_A * BT_NT) {
            int32_t ix[BT_PROW_A][8];
            Rt gv[BT_PROW_A][8];
            V xr[BT_PROW_A];
#pragma unroll
            for (int r = 0; r < BT_PROW_A; ++r) {
                const int e = e0 + r * BT_NT;
                const bool ok = e < vend;
                xr[r] = ok ? x[e] : mk<V>(0, 0);
                // the (<= 2) cells' bubbles: 4 consecutive rows from ab[u]
                int32_t b0[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) b0[u] = (ok && condensed) ? ab[u * n_loc + e] : -1;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    ix[r][u] = b0[u >> 2] >= 0 ? b0[u >> 2] + (u & 3) : -1;
                    gv[r][u] = (ok && condensed) ? (Rt)av[u * n_loc + e] : (Rt)0;
                }
            }
#pragma unroll
            for (int r = 0; r < BT_PROW_A; ++r) {
                const int e = e0 + r * BT_NT;
                Rt ar = xr[r].x, aim = xr[r].y;
                V xb[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) xb[u] = ix[r][u] >= 0 ? x[ix[r][u]] : mk<V>(0, 0);
                if (condensed) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        ar -= gv[r][u] * xb[u].x;
                        aim -= gv[r][u] * xb[u].y;
                    }
                }
                if (e < vend) vec[e - vbase] = mk<V>(ar, aim);
            }
        }
        bt_bar_consumers();
        int t = 0, tc = 0;                       // W / coupling tiles consumed
        for (int si = 0; si < nst; ++si) {
            const BtStep st = bt_step(rank, L, k, si, lv);
            const int m = lv[st.l].size, o = lv[st.l].start - vbase, ldm = bt_r4(m);
            // (b1) coupling term of the step (a backward step has none: its
            // GEMV input is x of level nb, final since the previous step)
            if (st.kind == 2) {
            } else if (st.cpl) {
                const int q = tc % BT_NC;
                const int nb = st.cpl == 1 ? st.l - 1 : st.l + 1;
                const int ob = lv[nb].start - vbase;
                const int nz = st.cpl == 1 ? lv[st.l].enz : lv[st.l].fnz;
                const int* P;
                const int* C;
                const F* Cv;
                if (cglob) {
                    const int64_t po = st.cpl == 1 ? lv[st.l].eptr : lv[st.l].fptr;
                    const int64_t qo = st.cpl == 1 ? lv[st.l].eoff : lv[st.l].foff;
                    P = cptr + po;
                    C = ccol + qo;
                    Cv = cval + qo;
                } else {
                    bt_wait<false>(&cfull[q], (unsigned)((tc / BT_NC) & 1), abort, err, wait_ns);
                    const unsigned char* buf = cslots + (size_t)q * cslot_bytes;
                    P = reinterpret_cast<const int*>(buf);
                    C = P + bt_r4(m + 1);
                    Cv = reinterpret_cast<const F*>(C + bt_r4(nz));
                }
                for (int i = tid; i < m; i += BT_NT) {
                    Rt ar = 0, aim = 0;
                    int pp = P[i];
                    const int pe = P[i + 1];
                    for (; pp + 4 <= pe; pp += 4) {       // four independent gathers in flight
                        int c[4];
                        Rt f[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) { c[u] = C[pp + u]; f[u] = (Rt)Cv[pp + u]; }
                        V v[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) v[u] = vec[ob + c[u]];
#pragma unroll
                        for (int u = 0; u < 4; ++u) { ar += f[u] * v[u].x; aim += f[u] * v[u].y; }
                    }
                    for (; pp < pe; ++pp) {
                        const Rt f = (Rt)Cv[pp];
                        const V v = vec[ob + C[pp]];
                        ar += f * v.x;
                        aim += f * v.y;
                    }
                    if (st.kind == 0) {
                        const V r = vec[o + i];
                        su[i] = mk<V>(r.x - ar, r.y - aim);
                    } else {
                        tx[i] = mk<V>(ar, aim);
                        prx[i] = mk<V>(ar, aim);
                    }
                }
                if (!cglob) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive_local(&cempty[q]);
                    ++tc;
                }
            } else {
                for (int i = tid; i < m; i += BT_NT) {
                    if (st.kind == 0) {
                        su[i] = vec[o + i];
                    } else {
                        tx[i] = mk<V>(0, 0);
                        prx[i] = mk<V>(0, 0);
                    }
                }
            }
            if (st.kind == 1) {
                // the peer's coupling term of the middle level arrives in rx
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(mapa_u32(&xbar[0], (unsigned)peer));
                bt_wait<true>(&xbar[0], 0u, abort, err, wait_ns);
                for (int i = tid; i < m; i += BT_NT) {
                    const V r = vec[o + i], a = tx[i], b = rx[i];
                    su[i] = mk<V>(r.x - a.x - b.x, r.y - a.y - b.y);
                }
            }
            if (st.kind != 2) bt_bar_consumers();
            // (b2)+(b3) y = W_l^T s (forward, middle) or H_l x_nb (backward) over
            // the rows [ra, rb) this rank streams
            const V* sin = st.kind == 2 ? vec + (lv[st.nb].start - vbase) : su;
            bt_gemv<BT_GQ, BT_GMAX, V, FW>(st, m, o, ldm, R, ns, slot_bytes, slots, full, empty, t, sin, vec, tx, pry,
                                           warp, lane, abort, err, wait_ns);
            if (st.kind == 1) {
                // x_k = own half + the peer's half (both complete once every
                // warp of both CTAs has written its outputs)
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(mapa_u32(&xbar[1], (unsigned)peer));
                bt_wait<true>(&xbar[1], 0u, abort, err, wait_ns);
                bt_bar_consumers();
                for (int i = tid; i < m; i += BT_NT) {
                    const V a = tx[i], b = ry[i];
                    vec[o + i] = mk<V>(a.x + b.x, a.y + b.y);
                }
            }
            bt_bar_consumers();
        }
        // write back: rank 0 levels 0..k, rank 1 levels k+1..L-1
        const int w0 = rank == 0 ? vbase : lv[k].start + lv[k].size;
        for (int e = w0 + tid; e < vend; e += BT_NT) y[e] = vec[e - vbase];
    }
    // (c) order 2: x_I = D^{-1} r_I - G^T x_E, once both ranks' edge values are in y
    cluster.sync();
    if (condensed) {
        const int64_t b0 = S.off + S.ne, nbub = S.n - S.ne;
        const int64_t half = (nbub + 1) / 2;
        const int64_t lo = b0 + (rank == 0 ? 0 : half), hi = b0 + (rank == 0 ? half : nbub);
        // BT_PROW_C rows per pass, as in (a)
        for (int64_t b0r = lo + tid; b0r < hi; b0r += BT_PROW_C * (int64_t)blockDim.x) {
            int32_t cix[BT_PROW_C][4], eix[BT_PROW_C][8];
            Rt cc[BT_PROW_C][4], ec[BT_PROW_C][8];
#pragma unroll
            for (int r = 0; r < BT_PROW_C; ++r) {
                const int64_t b = b0r + r * (int64_t)blockDim.x;
                const bool ok = b < hi;
                // the row's cell: its 4 bubbles are the rows cb..cb+3, its 8
                // edge rows are slot cell0 + (b - b0) / 4 of e8
                const int64_t q4 = b - b0, cb = b - (q4 & 3);
                const int32_t* ce = e8 + ((int64_t)S.cell0 + (q4 >> 2)) * 8;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    cix[r][j] = ok ? (int32_t)(cb + j) : -1;
                    cc[r][j] = ok ? (Rt)cv[j * n_loc + b] : (Rt)0;
                }
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    // the value is loaded whatever the index (it is masked
                    // below), so that both loads are in flight together
                    const int64_t e = ok ? (int64_t)ce[a] : -1;
                    eix[r][a] = (e >= S.off && e < S.off + S.ne) ? (int32_t)e : -1;
                    ec[r][a] = ok ? (Rt)ev[a * n_loc + b] : (Rt)0;
                }
            }
#pragma unroll
            for (int r = 0; r < BT_PROW_C; ++r) {
                const int64_t b = b0r + r * (int64_t)blockDim.x;
                V xb[4], xe[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) xb[j] = cix[r][j] >= 0 ? x[cix[r][j]] : mk<V>(0, 0);
#pragma unroll
                for (int a = 0; a < 8; ++a) xe[a] = eix[r][a] >= 0 ? y[eix[r][a]] : mk<V>(0, 0);
                Rt ar = 0, aim = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    ar += cc[r][j] * xb[j].x;
                    aim += cc[r][j] * xb[j].y;
                }
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    if (eix[r][a] >= 0) {
                        ar += ec[r][a] * xe[a].x;
                        aim += ec[r][a] * xe[a].y;
                    }
                }
                if (b < hi) y[b] = mk<V>(ar, aim);
            }
        }
    }
}

}  // namespace thm

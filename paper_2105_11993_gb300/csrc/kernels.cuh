// Device kernels of the solve phase (templated on vector/value precision).
#pragma once

#include "common.cuh"

namespace thm {

template <class V> struct VT;
template <> struct VT<double2> { using R = double; };
template <> struct VT<float2> { using R = float; };

template <class V>
__device__ __forceinline__ V mk(typename VT<V>::R a, typename VT<V>::R b);
template <> __device__ __forceinline__ double2 mk<double2>(double a, double b) { return make_double2(a, b); }
template <> __device__ __forceinline__ float2 mk<float2>(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// ---------------------------------------------------------------------------
// y = T_i x  (op 0: P + i(B_Gamma + B_Sigma))  or  K_i^loc x (op 2: P + i B_Gamma)
// SELL-32: one thread per row, slots column-major inside a slice (coalesced).
// ---------------------------------------------------------------------------
// 3-D: the face terms are not diagonal; their values (times kappa*omega) ride
// on the same SELL pattern (bvg: Gamma^inf, bvs: Sigma), non-null only then.
template <class V, class F>
__global__ void __launch_bounds__(256) k_spmv(int64_t n, const int64_t* __restrict__ slice_ptr,
                                              const int32_t* __restrict__ col, const F* __restrict__ val,
                                              const F* __restrict__ bg, const F* __restrict__ bs, int use_bs,
                                              const F* __restrict__ bvg, const F* __restrict__ bvs,
                                              const V* __restrict__ x, V* __restrict__ y) {
    using R = typename VT<V>::R;
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t sl = r >> 5;
    int lane = (int)(r & 31);
    int64_t base = slice_ptr[sl];
    int w = (int)((slice_ptr[sl + 1] - base) >> 5);
    R ar = 0, ai = 0;
    const int32_t* cp = col + base + lane;
    const F* vp = val + base + lane;
    if (bvg) {
        const F* gp = bvg + base + lane;
        const F* sp = bvs + base + lane;
        for (int t = 0; t < w; ++t) {
            int32_t c = __ldg(cp + (t << 5));
            R v = (R)__ldg(vp + (t << 5));
            R b = (R)__ldg(gp + (t << 5));
            if (use_bs) b += (R)__ldg(sp + (t << 5));
            V xv = x[c];
            ar += v * xv.x - b * xv.y;
            ai += v * xv.y + b * xv.x;
        }
    } else {
#pragma unroll 4
        for (int t = 0; t < w; ++t) {
            int32_t c = __ldg(cp + (t << 5));
            R v = (R)__ldg(vp + (t << 5));
            V xv = x[c];
            ar += v * xv.x;
            ai += v * xv.y;
        }
    }
    R b = (R)bg[r];
    if (use_bs) b += (R)bs[r];
    V xr = x[r];
    y[r] = mk<V>(ar - b * xr.y, ai + b * xr.x);
}

// ---------------------------------------------------------------------------
// y = P_i^{-1} x (Eq. 7: the same real P_i^{-1} on the real and on the
// imaginary part).  Grid (n_sub, 2): blockIdx.y picks the component, so the
// two independent real solves of one subdomain run on two SMs.
//   (a) order 2: r_E <- r_E - G r_I          (cell bubbles condensed)
//   (b) S^{-1} on the edge DOFs by the block-tridiagonal chain
//   (c) order 2: x_I = D^{-1} r_I - G^T x_E
// ---------------------------------------------------------------------------
template <class F, class R>
__device__ __forceinline__ R warp_dot(const F* __restrict__ a, const R* __restrict__ x, int n) {
    R acc = 0;
    for (int j = threadIdx.x & 31; j < n; j += 32) acc += (R)a[j] * x[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---- TMA 1-D bulk copies completing on an mbarrier (sm_90+ PTX) ----------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// bytes must be a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// Bounded wait for the given phase parity; false after the iteration limit
// (each try_wait itself suspends for a bounded, hardware-defined time).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Copy n 4-byte words (16-byte aligned source, readable up to the next 16
// bytes) into shared memory with cp.async, cooperatively.
__device__ __forceinline__ void stage_words(void* dst, const void* __restrict__ src, int64_t words) {
    const int64_t chunks = (words + 3) / 4;
    const char* s = reinterpret_cast<const char*>(src);
    char* d = reinterpret_cast<char*>(dst);
    for (int64_t q = threadIdx.x; q < chunks; q += blockDim.x) cp_async16(d + 16 * q, s + 16 * q);
}

// Tile stream of one block-tridiagonal apply: for each level of the forward
// sweep (l = 0..L-1) and of the backward sweep (l = L-2..0) one coupling
// tile (the level's CSR block to its neighbour) followed by row tiles of W_l.
struct TileCursor {
    int dir;   // 0 forward, 1 backward, 2 finished
    int l;
    int r0;    // -1: coupling tile; otherwise first row of a W tile
};

// Row-tile height of a level of m rows: at most R rows, tiles of nearly
// equal height, every tile start a multiple of 4 rows (16-byte aligned rows).
__device__ __forceinline__ int tile_rows(int m, int R) {
    const int nt = (m + R - 1) / R;
    return (((m + nt - 1) / nt) + 3) / 4 * 4;
}

__device__ __forceinline__ void tile_next(TileCursor& c, int nlev, const int* msz, int R) {
    if (c.r0 < 0) { c.r0 = 0; return; }
    c.r0 += tile_rows(msz[c.l], R);
    if (c.r0 < msz[c.l]) return;
    c.r0 = -1;
    if (c.dir == 0) {
        if (c.l + 1 < nlev) { c.l++; return; }
        c.dir = 1;
        c.l = nlev - 2;
        if (c.l < 0) c.dir = 2;
        return;
    }
    c.l--;
    if (c.l < 0) c.dir = 2;
}

constexpr int BT_NG = 4;        // column groups of the block GEMV
constexpr int BT_MAXO = 8;      // outputs per thread: level blocks up to 8 * 512 / BT_NG = 1024 rows

// x = P_i^{-1} y for every subdomain (Eq. 7: the same real P_i^{-1} on the
// real and on the imaginary part).  Grid (n_sub, 2): blockIdx.y picks the
// component, so the two independent real solves of a subdomain run on two
// SMs.  The subdomain's edge vector stays in shared memory through
//   (a) order 2: r_E <- r_E - G r_I               (bubbles condensed per cell)
//   (b) S^{-1} r_E by the block-tridiagonal chain: z_l = W_l (r_l - E_l z_{l-1}),
//       then x_l = z_l - W_l F_l x_{l+1}.  W_l streams through a ring of
//       nslot shared-memory tiles of R rows, nslot-2 tiles ahead of use
//       (cp.async groups), so HBM latency is covered without a spin-wait.
//   (c) order 2: x_I = D^{-1} r_I - G^T x_E
template <class V, class F>
__global__ void __launch_bounds__(512) k_bt_apply(const Sub* __restrict__ subs, const Level* __restrict__ levels,
                                                  const F* __restrict__ fac, const int32_t* __restrict__ cptr,
                                                  const int32_t* __restrict__ ccol, const F* __restrict__ cval,
                                                  int64_t n_loc, int condensed, const int32_t* __restrict__ ai,
                                                  const F* __restrict__ av, const int32_t* __restrict__ ci,
                                                  const F* __restrict__ cv, const int32_t* __restrict__ ei,
                                                  const F* __restrict__ ev, int R, int nslot, int slot_bytes,
                                                  int max_ne, int max_m, int max_lev, int* __restrict__ err,
                                                  const V* __restrict__ xin, V* __restrict__ yout) {
    using R_t = typename VT<V>::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_abort;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);                    // [nslot]
    unsigned char* slots = smem_raw + ((nslot * 8 + 15) / 16) * 16;
    R_t* vec = reinterpret_cast<R_t*>(slots + (size_t)nslot * slot_bytes);
    R_t* su = vec + ((max_ne + 3) / 4) * 4;
    R_t* part = su + ((max_m + 3) / 4) * 4;                            // [BT_NG][max_m] partial sums
    int* msz = reinterpret_cast<int*>(part + BT_NG * (((max_m + 3) / 4) * 4));   // [max_lev] level sizes
    int* mst = msz + max_lev;                                          // level starts (relative)
    int* enz = mst + max_lev;                                          // coupling entries E, F
    int* fnz = enz + max_lev;
    long long* offw = reinterpret_cast<long long*>(fnz + max_lev);   // 16-byte aligned: 4*max_lev ints precede
    long long* eptr = offw + max_lev;
    long long* eoff = eptr + max_lev;
    long long* fptr = eoff + max_lev;
    long long* foff = fptr + max_lev;
    const Sub S = subs[blockIdx.x];
    const int comp = blockIdx.y;
    const R_t* x = reinterpret_cast<const R_t*>(xin) + comp;     // stride 2
    R_t* y = reinterpret_cast<R_t*>(yout) + comp;
    // thread groups of the block GEMV, sized to the widest level: tpg threads
    // (a multiple of 32, >= max_m when it fits) own outputs i0, i0+tpg, ...;
    // ng groups split the rows of each tile
    const int tpg = min((int)blockDim.x, ((max_m + 31) / 32) * 32);
    const int ng = min(BT_NG, (int)blockDim.x / tpg);
    const int g = threadIdx.x / tpg, i0 = threadIdx.x % tpg;
    const bool in_group = g < ng;
    R_t acc[BT_MAXO];
    for (int l = threadIdx.x; l < S.nlev; l += blockDim.x) {
        const Level L = levels[S.lev0 + l];
        msz[l] = L.size;
        mst[l] = (int)(L.start - S.off);
        enz[l] = L.enz; fnz[l] = L.fnz;
        offw[l] = L.offW; eptr[l] = L.eptr; eoff[l] = L.eoff; fptr[l] = L.fptr; foff[l] = L.foff;
    }
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int q = 0; q < nslot; ++q) mbar_init(&bars[q], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // producer (thread 0): one TMA bulk copy per W tile, three per coupling tile
    auto issue = [&](const TileCursor& c, int t) {
        if (threadIdx.x != 0 || c.dir == 2) return;
        const int q = t % nslot;
        unsigned char* dst = slots + (size_t)q * slot_bytes;
        const int m = msz[c.l];
        fence_proxy_async();
        if (c.r0 < 0) {
            const bool fwd = c.dir == 0;
            const int64_t po = fwd ? eptr[c.l] : fptr[c.l], qo = fwd ? eoff[c.l] : foff[c.l];
            const int nz = fwd ? enz[c.l] : fnz[c.l];
            const unsigned pb = (unsigned)(((m + 1) * 4 + 15) / 16 * 16);
            const unsigned cb = (unsigned)((nz * 4 + 15) / 16 * 16);
            const unsigned vb = (unsigned)((nz * (int)sizeof(F) + 15) / 16 * 16);
            mbar_expect_tx(&bars[q], pb + cb + vb);
            tma_load_1d(dst, cptr + po, pb, &bars[q]);
            if (cb) tma_load_1d(dst + pb, ccol + qo, cb, &bars[q]);
            if (vb) tma_load_1d(dst + pb + cb, cval + qo, vb, &bars[q]);
        } else {
            const int nr = min(tile_rows(m, R), m - c.r0);
            const unsigned wb = (unsigned)(((int64_t)nr * m * (int64_t)sizeof(F) + 15) / 16 * 16);
            mbar_expect_tx(&bars[q], wb);
            tma_load_1d(dst, fac + offw[c.l] + (int64_t)c.r0 * m, wb, &bars[q]);
        }
    };

    // prologue: fill the ring
    TileCursor prod{S.nlev > 0 ? 0 : 2, 0, -1};
    int tp = 0;
    for (int q = 0; q < nslot && prod.dir < 2; ++q) {
        issue(prod, tp++);
        tile_next(prod, S.nlev, msz, R);
    }
    // (a)
    for (int64_t e = threadIdx.x; e < S.ne; e += blockDim.x) {
        const int64_t r = S.off + e;
        R_t acc = x[2 * r];
        if (condensed) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc -= (R_t)av[u * n_loc + r] * x[2 * (int64_t)ai[u * n_loc + r]];
        }
        vec[e] = acc;
    }
    __syncthreads();
    // (b)
    TileCursor cur{S.nlev > 0 ? 0 : 2, 0, -1};
    int t = 0;
    for (; cur.dir < 2; ++t) {
        if (!mbar_wait(&bars[t % nslot], (unsigned)((t / nslot) & 1))) {
            atomicExch(err, 1);
            s_abort = 1;
        }
        const unsigned char* buf = slots + (size_t)(t % nslot) * slot_bytes;
        const int m = msz[cur.l];
        const int o = mst[cur.l];
        if (cur.r0 < 0) {
            const int* P = reinterpret_cast<const int*>(buf);
            const int pw = ((m + 1 + 3) / 4) * 4;
            const int* C = P + pw;
            const int nz = cur.dir == 0 ? enz[cur.l] : fnz[cur.l];
            const F* Vv = reinterpret_cast<const F*>(C + ((nz + 3) / 4) * 4);
            if (cur.dir == 0) {
                const int op = cur.l > 0 ? mst[cur.l - 1] : 0;
                for (int i = threadIdx.x; i < m; i += blockDim.x) {
                    R_t acc = vec[o + i];
                    for (int p = P[i]; p < P[i + 1]; ++p) acc -= (R_t)Vv[p] * vec[op + C[p]];
                    su[i] = acc;
                }
            } else {
                const int on = mst[cur.l + 1];
                for (int i = threadIdx.x; i < m; i += blockDim.x) {
                    R_t acc = 0;
                    for (int p = P[i]; p < P[i + 1]; ++p) acc += (R_t)Vv[p] * vec[on + C[p]];
                    su[i] = acc;
                }
            }
        } else {
            // rows j0..j0+nr of W_l; W_l = S_l^{-1} is symmetric, so these rows
            // are also columns: y_i += sum_{j in tile} W[j][i] s_j.  Thread
            // (group g, lane-in-group i0) owns outputs i0, i0+TPG, ... and the
            // tile rows j0+g, j0+g+BT_NG, ...; consecutive threads read
            // consecutive words of a row (no bank conflicts), s_j is a broadcast.
            const F* Wt = reinterpret_cast<const F*>(buf);
            const int j0 = cur.r0;
            const int nr = min(tile_rows(m, R), m - j0);
            const int nout = (m - i0 + tpg - 1) / tpg;     // outputs of this thread (i0 < m)
            if (j0 == 0)
#pragma unroll
                for (int k = 0; k < BT_MAXO; ++k) acc[k] = 0;
            if (in_group && i0 < m) {
                if (nout == 1) {
                    R_t a0 = acc[0];
                    for (int jj = g; jj < nr; jj += ng) a0 += (R_t)Wt[(int64_t)jj * m + i0] * su[j0 + jj];
                    acc[0] = a0;
                } else {
                    for (int jj = g; jj < nr; jj += ng) {
                        const R_t sj = su[j0 + jj];
                        const F* wr = Wt + (int64_t)jj * m + i0;
#pragma unroll
                        for (int k = 0; k < BT_MAXO; ++k)
                            if (k < nout) acc[k] += (R_t)wr[k * tpg] * sj;
                    }
                }
            }
            if (j0 + nr >= m) {                // last tile of the level: combine the groups
                if (in_group)
#pragma unroll
                    for (int k = 0; k < BT_MAXO; ++k) {
                        const int i = i0 + k * tpg;
                        if (i < m) part[g * ((max_m + 3) / 4 * 4) + i] = acc[k];
                    }
                __syncthreads();
                for (int i = threadIdx.x; i < m; i += blockDim.x) {
                    R_t v = 0;
                    for (int q = 0; q < ng; ++q) v += part[q * ((max_m + 3) / 4 * 4) + i];
                    if (cur.dir == 0) vec[o + i] = v;
                    else vec[o + i] -= v;
                }
            }
        }
        __syncthreads();                       // slot t%nslot free, vec/su writes visible
        if (s_abort) break;
        issue(prod, tp);                       // refill the freed slot
        if (prod.dir < 2) { ++tp; tile_next(prod, S.nlev, msz, R); }
        tile_next(cur, S.nlev, msz, R);
    }
    if (s_abort) {
        // a copy did not arrive: wait (bounded) for the ones in flight, then leave
        if (threadIdx.x == 0)
            for (int q = t + 1; q < tp; ++q) mbar_wait(&bars[q % nslot], (unsigned)((q / nslot) & 1));
        return;
    }
    // (c) and write-back
    for (int64_t e = threadIdx.x; e < S.ne; e += blockDim.x) y[2 * (S.off + e)] = vec[e];
    if (condensed)
        for (int64_t b = S.off + S.ne + threadIdx.x; b < S.off + S.n; b += blockDim.x) {
            R_t acc = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) acc += (R_t)cv[j * n_loc + b] * x[2 * (int64_t)ci[j * n_loc + b]];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                int64_t e = (int64_t)ei[a * n_loc + b] - S.off;
                R_t tt = (e >= 0 && e < S.ne) ? vec[e] : (R_t)0;
                acc += (R_t)ev[a * n_loc + b] * tt;
            }
            y[2 * b] = acc;
        }
}

// ---------------------------------------------------------------------------
// Segmented reductions for the batched Arnoldi process.  A chunk lies inside
// one segment (subdomain); per-chunk partials are summed per segment in a
// fixed order, so every dot product is deterministic.
// ---------------------------------------------------------------------------
constexpr int KT = 256;                       // threads per chunk block
constexpr int EPT = CHUNK / KT;               // elements per thread

template <class V>
__global__ void __launch_bounds__(KT) k_chunk_dots(const Chunk* __restrict__ chunks, const V* __restrict__ basis,
                                                   int64_t ld, int nk, const V* __restrict__ w,
                                                   double2* __restrict__ partial, int ldp) {
    using R = typename VT<V>::R;
    extern __shared__ double2 sred[];          // [nk][KT/32]
    const Chunk c = chunks[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    V wr[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        int64_t e = c.begin + threadIdx.x + (int64_t)q * KT;
        wr[q] = e < c.end ? w[e] : mk<V>(0, 0);
    }
    const bool full = c.end - c.begin == CHUNK;
    int k = 0;
    for (; k < nk; ++k) {
        const V* vk = basis + (int64_t)k * ld;
        R ar = 0, ai = 0;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            int64_t e = c.begin + threadIdx.x + (int64_t)q * KT;
            if (full || e < c.end) {
                V v = vk[e];
                ar += v.x * wr[q].x + v.y * wr[q].y;       // conj(v) * w
                ai += v.x * wr[q].y - v.y * wr[q].x;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ar += __shfl_down_sync(0xffffffffu, ar, o);
            ai += __shfl_down_sync(0xffffffffu, ai, o);
        }
        if (lane == 0) sred[k * (KT / 32) + warp] = make_double2((double)ar, (double)ai);
    }
    __syncthreads();
    for (int kk = threadIdx.x; kk < nk; kk += KT) {
        double2 s = make_double2(0, 0);
        for (int q = 0; q < KT / 32; ++q) s = cadd(s, sred[kk * (KT / 32) + q]);
        partial[(int64_t)blockIdx.x * ldp + kk] = s;
    }
}

// w -= sum_k h[seg][k] basis_k ;  optionally per-chunk ||w||^2
template <class V>
__global__ void __launch_bounds__(KT) k_chunk_update(const Chunk* __restrict__ chunks, const V* __restrict__ basis,
                                                     int64_t ld, int nk, const double2* __restrict__ h, int ldh,
                                                     V* __restrict__ w, double* __restrict__ nrm_part) {
    using R = typename VT<V>::R;
    extern __shared__ double2 sh[];            // [nk] coefficients of this segment
    __shared__ double sw[KT / 32];
    const Chunk c = chunks[blockIdx.x];
    for (int k = threadIdx.x; k < nk; k += KT) sh[k] = h[(int64_t)c.seg * ldh + k];
    __syncthreads();
    const bool full = c.end - c.begin == CHUNK;
    R xr[EPT], xi[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        int64_t e = c.begin + threadIdx.x + (int64_t)q * KT;
        V a = (full || e < c.end) ? w[e] : mk<V>(0, 0);
        xr[q] = a.x;
        xi[q] = a.y;
    }
    for (int k = 0; k < nk; ++k) {             // basis index outer: EPT independent loads per step
        const V* vk = basis + (int64_t)k * ld;
        const R hr = (R)sh[k].x, hi = (R)sh[k].y;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            int64_t e = c.begin + threadIdx.x + (int64_t)q * KT;
            if (full || e < c.end) {
                V v = vk[e];
                xr[q] -= hr * v.x - hi * v.y;
                xi[q] -= hr * v.y + hi * v.x;
            }
        }
    }
    R nr = 0;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        int64_t e = c.begin + threadIdx.x + (int64_t)q * KT;
        if (full || e < c.end) {
            w[e] = mk<V>(xr[q], xi[q]);
            nr += xr[q] * xr[q] + xi[q] * xi[q];
        }
    }
    if (nrm_part) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nr += __shfl_down_sync(0xffffffffu, nr, o);
        if (lane == 0) sw[warp] = (double)nr;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int q = 0; q < KT / 32; ++q) s += sw[q];
            nrm_part[blockIdx.x] = s;
        }
    }
}

template <class V>
__global__ void __launch_bounds__(KT) k_chunk_norm2(const Chunk* __restrict__ chunks, const V* __restrict__ x,
                                                    double* __restrict__ nrm_part) {
    using R = typename VT<V>::R;
    __shared__ double sw[KT / 32];
    const Chunk c = chunks[blockIdx.x];
    R nr = 0;
    for (int64_t e = c.begin + threadIdx.x; e < c.end; e += KT) {
        V v = x[e];
        nr += v.x * v.x + v.y * v.y;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nr += __shfl_down_sync(0xffffffffu, nr, o);
    if (lane == 0) sw[warp] = (double)nr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int q = 0; q < KT / 32; ++q) s += sw[q];
        nrm_part[blockIdx.x] = s;
    }
}

// out[seg][k] (+)= sum over the segment's chunks of partial[chunk][k]
__global__ void k_seg_reduce(int nseg, const int32_t* __restrict__ seg_ch, const double2* __restrict__ partial,
                             int ldp, int nk, double2* __restrict__ out, int ldo, int accumulate);
__global__ void k_seg_reduce_real(int nseg, const int32_t* __restrict__ seg_ch, const double* __restrict__ part,
                                  double* __restrict__ out);

// scale: x[e] = (beta[seg] > 0) ? r[e] / beta[seg] : 0
template <class V>
__global__ void k_chunk_scale(const Chunk* __restrict__ chunks, const V* __restrict__ r,
                              const double* __restrict__ beta, V* __restrict__ x) {
    using R = typename VT<V>::R;
    const Chunk c = chunks[blockIdx.x];
    double b = beta[c.seg];
    R inv = b > 0 ? (R)(1.0 / b) : (R)0;
    for (int64_t e = c.begin + threadIdx.x; e < c.end; e += blockDim.x) {
        V v = r[e];
        x[e] = mk<V>(v.x * inv, v.y * inv);
    }
}

// t[e] = sum_{k < kused[seg]} y[seg][k] basis_k[e]
template <class V>
__global__ void __launch_bounds__(KT) k_chunk_combine(const Chunk* __restrict__ chunks, const V* __restrict__ basis,
                                                      int64_t ld, const int* __restrict__ kused,
                                                      const double2* __restrict__ y, int ldy, V* __restrict__ t) {
    using R = typename VT<V>::R;
    const Chunk c = chunks[blockIdx.x];
    const int nk = kused[c.seg];
    const double2* yy = y + (int64_t)c.seg * ldy;
    for (int64_t e = c.begin + threadIdx.x; e < c.end; e += KT) {
        R xr = 0, xi = 0;
        for (int k = 0; k < nk; ++k) {
            V v = basis[(int64_t)k * ld + e];
            R a = (R)yy[k].x, b = (R)yy[k].y;
            xr += a * v.x - b * v.y;
            xi += a * v.y + b * v.x;
        }
        t[e] = mk<V>(xr, xi);
    }
}

template <class V>
__global__ void k_axpy(int64_t n, const V* __restrict__ a, V* __restrict__ x) {  // x += a
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        V u = x[i], v = a[i];
        x[i] = mk<V>(u.x + v.x, u.y + v.y);
    }
}

template <class V>
__global__ void k_sub(int64_t n, const V* __restrict__ a, const V* __restrict__ b, V* __restrict__ out) {  // a - b
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        V u = a[i], v = b[i];
        out[i] = mk<V>(u.x - v.x, u.y - v.y);
    }
}

template <class A, class B>
__global__ void k_convert(int64_t n, const A* __restrict__ a, B* __restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        A u = a[i];
        b[i].x = u.x;
        b[i].y = u.y;
    }
}

}  // namespace thm

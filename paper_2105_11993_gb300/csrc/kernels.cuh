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
// Column indices: int32 local indices, or (CI = uint16_t) indices relative
// to the row's subdomain (subs[row_seg[r]].off added back), half the bytes of
// the index stream.
template <class V, class F, class CI = int32_t>
__global__ void __launch_bounds__(256) k_spmv(int64_t n, const int64_t* __restrict__ slice_ptr,
                                              const CI* __restrict__ col, const Sub* __restrict__ subs,
                                              const F* __restrict__ val,
                                              const F* __restrict__ bg, const F* __restrict__ bs, int use_bs,
                                              const F* __restrict__ bvg, const F* __restrict__ bvs,
                                              const V* __restrict__ x, V* __restrict__ y,
                                              const int32_t* __restrict__ row_seg, const int* __restrict__ act,
                                              unsigned long long* __restrict__ work) {
    using R = typename VT<V>::R;
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // a converged subdomain's rows are not needed
    const bool on = r < n && !(act && !act[row_seg[r < n ? r : 0]]);
    if (work) {                                // rows processed (uniform branch: every thread reaches the count)
        const int cnt = __syncthreads_count(on);
        if (threadIdx.x == 0 && cnt) atomicAdd(work, (unsigned long long)cnt);
    }
    if (!on) return;
    int64_t sl = r >> 5;
    int lane = (int)(r & 31);
    int64_t base = slice_ptr[sl];
    int w = (int)((slice_ptr[sl + 1] - base) >> 5);
    R ar = 0, ai = 0;
    const CI* cp = col + base + lane;
    const V* xs = x;                           // column origin
    if constexpr (sizeof(CI) == 2) xs = x + subs[row_seg[r]].off;
    const F* vp = val + base + lane;
    if (bvg) {
        const F* gp = bvg + base + lane;
        const F* sp = bvs + base + lane;
        for (int t = 0; t < w; ++t) {
            int32_t c = (int32_t)__ldg(cp + (t << 5));
            R v = (R)__ldg(vp + (t << 5));
            R b = (R)__ldg(gp + (t << 5));
            if (use_bs) b += (R)__ldg(sp + (t << 5));
            V xv = xs[c];
            ar += v * xv.x - b * xv.y;
            ai += v * xv.y + b * xv.x;
        }
    } else {
        // slots in groups of 8: the 8 index and value loads, then the 8
        // gathers of x, are in flight together
        for (int t0 = 0; t0 < w; t0 += 8) {
            int32_t c[8];
            R v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                c[u] = (int32_t)(r - (xs - x));    // own row (its x is read below anyway)
                v[u] = 0;
                if (t0 + u < w) {
                    c[u] = (int32_t)__ldg(cp + ((t0 + u) << 5));
                    v[u] = (R)__ldg(vp + ((t0 + u) << 5));
                }
            }
            V xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) xv[u] = xs[c[u]];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                ar += v[u] * xv[u].x;
                ai += v[u] * xv[u].y;
            }
        }
    }
    R b = (R)bg[r];
    if (use_bs) b += (R)bs[r];
    V xr = x[r];
    y[r] = mk<V>(ar - b * xr.y, ai + b * xr.x);
}

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

// ---------------------------------------------------------------------------
// Segmented reductions for the batched Arnoldi process.  A chunk lies inside
// one segment (subdomain); per-chunk partials are summed per segment in a
// fixed order, so every dot product is deterministic.
// ---------------------------------------------------------------------------
constexpr int KT = 256;                       // threads per chunk block
constexpr int EPT = CHUNK / KT;               // elements per thread

// The last block of a segment to finish (per-segment arrival counter) sums
// the segment's per-chunk partials in chunk order, so the result does not
// depend on which block finishes last, and resets the counter for the next
// launch.  Partials of other blocks are read through L2 (__ldcg).
__device__ __forceinline__ bool last_block_of_segment(int seg, const int32_t* __restrict__ seg_ch, int* cnt) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&cnt[seg], 1) == seg_ch[seg + 1] - seg_ch[seg] - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x == 0) cnt[seg] = 0;
    }
    return s_last != 0;
}

// h[seg][k] = sum over the segment's chunks of v_k^H w (FP64), k < nk.
// reset (optional): an int the first block sets to 0 (the active-segment
// count that the Givens step of the same Arnoldi step accumulates).
// h[seg][k] = v_k^H w for the chunk c of a block whose threads hold w in
// wr (EPT elements each); the last block of the segment writes h.
template <class V>
__device__ __forceinline__ void chunk_dots_body(const Chunk& c, const V* __restrict__ basis, int64_t ld, int nk,
                                                const V (&wr)[EPT], double2* __restrict__ partial, int ldp,
                                                const int32_t* __restrict__ seg_ch, int* __restrict__ cnt,
                                                double2* __restrict__ h, int ldh, double2* sred);

template <class V>
__global__ void __launch_bounds__(KT) k_chunk_dots(const Chunk* __restrict__ chunks, const V* __restrict__ basis,
                                                   int64_t ld, int nk, const V* __restrict__ w,
                                                   double2* __restrict__ partial, int ldp,
                                                   const int* __restrict__ act, const int32_t* __restrict__ seg_ch,
                                                   int* __restrict__ cnt, double2* __restrict__ h, int ldh,
                                                   int* __restrict__ reset, unsigned long long* __restrict__ work) {
    extern __shared__ double2 sred[];          // [nk][KT/32]
    if (reset && blockIdx.x == 0 && threadIdx.x == 0) *reset = 0;
    const Chunk c = chunks[blockIdx.x];
    if (act && !act[c.seg]) return;            // converged segment: its partials are not read
    if (work && threadIdx.x == 0) atomicAdd(work, (unsigned long long)((nk + 1) * (c.end - c.begin) * sizeof(V)));
    V wr[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        int64_t e = c.begin + threadIdx.x + (int64_t)q * KT;
        wr[q] = e < c.end ? w[e] : mk<V>(0, 0);
    }
    chunk_dots_body<V>(c, basis, ld, nk, wr, partial, ldp, seg_ch, cnt, h, ldh, sred);
}

template <class V>
__device__ __forceinline__ void chunk_dots_body(const Chunk& c, const V* __restrict__ basis, int64_t ld, int nk,
                                                const V (&wr)[EPT], double2* __restrict__ partial, int ldp,
                                                const int32_t* __restrict__ seg_ch, int* __restrict__ cnt,
                                                double2* __restrict__ h, int ldh, double2* sred) {
    using R = typename VT<V>::R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool full = c.end - c.begin == CHUNK;
    // basis vectors in blocks of KB: their KB * EPT loads are issued together,
    // so a block of vectors costs one memory latency instead of KB
    constexpr int KB = 4;
    for (int k0 = 0; k0 < nk; k0 += KB) {
        V v[KB][EPT];
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            const V* vk = basis + (int64_t)(k0 + b) * ld;
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int64_t e = c.begin + threadIdx.x + (int64_t)q * KT;
                v[b][q] = mk<V>(0, 0);
                if (k0 + b < nk && (full || e < c.end)) v[b][q] = vk[e];
            }
        }
        R ar[KB], ai[KB];
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            ar[b] = 0;
            ai[b] = 0;
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                ar[b] += v[b][q].x * wr[q].x + v[b][q].y * wr[q].y;       // conj(v) * w
                ai[b] += v[b][q].x * wr[q].y - v[b][q].y * wr[q].x;
            }
        }
        // a warp sums its 4 * 32 products in the vector precision; from the
        // cross-warp sum on every sum is FP64 (FP64 shuffles at the warp level
        // cost 2.7x the kernel time on this part, measured)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int b = 0; b < KB; ++b) {
                ar[b] += __shfl_down_sync(0xffffffffu, ar[b], o);
                ai[b] += __shfl_down_sync(0xffffffffu, ai[b], o);
            }
        if (lane == 0)
#pragma unroll
            for (int b = 0; b < KB; ++b)
                if (k0 + b < nk) sred[(k0 + b) * (KT / 32) + warp] = make_double2((double)ar[b], (double)ai[b]);
    }
    __syncthreads();
    for (int kk = threadIdx.x; kk < nk; kk += KT) {
        double2 s = make_double2(0, 0);
        for (int q = 0; q < KT / 32; ++q) s = cadd(s, sred[kk * (KT / 32) + q]);
        partial[(int64_t)blockIdx.x * ldp + kk] = s;
    }
    if (!last_block_of_segment(c.seg, seg_ch, cnt)) return;
    for (int kk = threadIdx.x; kk < nk; kk += KT) {
        double2 s = make_double2(0, 0);
        for (int cc = seg_ch[c.seg]; cc < seg_ch[c.seg + 1]; ++cc) {
            const double2 p = __ldcg(&partial[(int64_t)cc * ldp + kk]);
            s.x += p.x;
            s.y += p.y;
        }
        h[(int64_t)c.seg * ldh + kk] = s;
    }
}

// w -= sum_k h[seg][k] basis_k ;  optionally per-chunk ||w||^2
template <class V>
__device__ __forceinline__ void chunk_update_body(const Chunk& c, const V* __restrict__ basis, int64_t ld, int nk,
                                                  const double2* __restrict__ h, int ldh, V* __restrict__ w,
                                                  double* __restrict__ nrm_part, double2* sh, V* wout = nullptr);


template <class V>
__device__ __forceinline__ void chunk_update_body(const Chunk& c, const V* __restrict__ basis, int64_t ld, int nk,
                                                  const double2* __restrict__ h, int ldh, V* __restrict__ w,
                                                  double* __restrict__ nrm_part, double2* sh, V* wout) {
    using R = typename VT<V>::R;
    __shared__ double sw[KT / 32];
    // the coefficients in the vector precision, rounded once per block (a
    // double-to-float conversion per use would run on the slow FP64 path)
    V* shv = reinterpret_cast<V*>(sh);
    for (int k = threadIdx.x; k < nk; k += KT) {
        const double2 hk = h[(int64_t)c.seg * ldh + k];
        shv[k] = mk<V>((R)hk.x, (R)hk.y);
    }
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
    // basis vectors in blocks of KB: KB * EPT independent loads in flight
    constexpr int KB = 4;
    for (int k0 = 0; k0 < nk; k0 += KB) {
        V v[KB][EPT];
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            const V* vk = basis + (int64_t)(k0 + b) * ld;
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int64_t e = c.begin + threadIdx.x + (int64_t)q * KT;
                v[b][q] = mk<V>(0, 0);
                if (k0 + b < nk && (full || e < c.end)) v[b][q] = vk[e];
            }
        }
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            const int kk = min(k0 + b, nk - 1);
            const V hv = shv[kk];
            const R hr = k0 + b < nk ? hv.x : (R)0, hi = k0 + b < nk ? hv.y : (R)0;
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                xr[q] -= hr * v[b][q].x - hi * v[b][q].y;
                xi[q] -= hr * v[b][q].y + hi * v[b][q].x;
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
        if (wout) wout[q] = (full || e < c.end) ? mk<V>(xr[q], xi[q]) : mk<V>(0, 0);
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

// First Gram-Schmidt update and second projection in one pass over the
// chunk: w <- w - V h1 (written back), then h2 = V^H w from the updated
// values still in registers.  The block rereads its basis slab right after
// the update, while it is in L2, so V is streamed from DRAM once for both.
template <class V>
__global__ void __launch_bounds__(KT) k_update_dots(const Chunk* __restrict__ chunks, const V* __restrict__ basis,
                                                    int64_t ld, int nk, const double2* __restrict__ h1, int ldh,
                                                    V* __restrict__ w, double2* __restrict__ partial, int ldp,
                                                    const int* __restrict__ act, const int32_t* __restrict__ seg_ch,
                                                    int* __restrict__ cnt, double2* __restrict__ h2,
                                                    unsigned long long* __restrict__ work) {
    extern __shared__ double2 sh[];            // [nk] coefficients, then [nk][KT/32] warp sums
    const Chunk c = chunks[blockIdx.x];
    if (act && !act[c.seg]) return;
    // the basis twice, w read and written
    if (work && threadIdx.x == 0) atomicAdd(work, (unsigned long long)((2 * nk + 2) * (c.end - c.begin) * sizeof(V)));
    V wr[EPT];
    chunk_update_body<V>(c, basis, ld, nk, h1, ldh, w, nullptr, sh, wr);
    __syncthreads();                           // sh is reused for the warp sums
    chunk_dots_body<V>(c, basis, ld, nk, wr, partial, ldp, seg_ch, cnt, h2, ldh, sh);
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

__global__ void k_seg_reduce_real(int nseg, const int32_t* __restrict__ seg_ch, const double* __restrict__ part,
                                  double* __restrict__ out);

// scale: x[e] = (beta[seg] > 0) ? r[e] / beta[seg] : 0
template <class V>
__global__ void k_chunk_scale(const Chunk* __restrict__ chunks, const V* __restrict__ r,
                              const double* __restrict__ beta, V* __restrict__ x, const int* __restrict__ act) {
    using R = typename VT<V>::R;
    __shared__ R s_inv;
    const Chunk c = chunks[blockIdx.x];
    if (act && !act[c.seg]) return;
    if (threadIdx.x == 0) {                    // one FP64 division per block, not per thread
        const double b = beta[c.seg];
        s_inv = b > 0 ? (R)(1.0 / b) : (R)0;
    }
    __syncthreads();
    const R inv = s_inv;
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
    extern __shared__ double2 ys_raw[];        // [ldy] y of this segment in the vector precision
    V* ys = reinterpret_cast<V*>(ys_raw);
    const Chunk c = chunks[blockIdx.x];
    const int nk = kused[c.seg];
    const double2* yy = y + (int64_t)c.seg * ldy;
    for (int k = threadIdx.x; k < nk; k += KT) ys[k] = mk<V>((R)yy[k].x, (R)yy[k].y);
    __syncthreads();
    for (int64_t e = c.begin + threadIdx.x; e < c.end; e += KT) {
        R xr = 0, xi = 0;
        for (int k = 0; k < nk; ++k) {
            const V v = basis[(int64_t)k * ld + e], a = ys[k];
            xr += a.x * v.x - a.y * v.y;
            xi += a.x * v.y + a.y * v.x;
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

}  // namespace thm

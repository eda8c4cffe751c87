// thm_residual_noalloc: the FP64 true residual ||f - K u|| and ||f|| of a
// field u without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the moment they want a
// residual check: a host program that hands all device memory to its own
// pool allocator up front (cudaMalloc then fails), or a time-critical loop
// that must not call cudaMalloc/cudaFree because they synchronise the whole
// device.  The regular path (thm_ddm_solve's refinement check) allocates its
// work vectors lazily.
//
// The only scratch is the file-scope array below: per-block partial sums of
// |f - K u|^2 and |f|^2.  Each GPU that loads this library holds those 64 KB
// until the process exits.
#include <mutex>

#include "common.cuh"

namespace thm {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_BLOCK = 1024;                      // global DOFs per block
constexpr int NA_MAX_BLOCKS = 4096;                     // => n_dof <= 4,194,304
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_na_scratch[2 * NA_MAX_BLOCKS];

// Per global DOF d (free DOFs have local copies, Dirichlet DOFs none):
//   f_d = sum over copies c of f_loc[c]
//   r_d = sum over copies c of (f_loc[c] - (K_i^loc u)[c]),  u gathered through loc_gdof
// Block b writes its partial sums to scratch[b] and scratch[NA_MAX_BLOCKS + b].
__global__ void __launch_bounds__(NA_THREADS) k_na_residual(
    int64_t n_dof, const int64_t* __restrict__ copy_ptr, const int32_t* __restrict__ copy_idx,
    const int64_t* __restrict__ loc_gdof, const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
    const double* __restrict__ val, const double* __restrict__ bg, const double* __restrict__ bvg,
    const double2* __restrict__ f_loc,
    const double2* __restrict__ u, double* __restrict__ scratch) {
    __shared__ double sr[NA_THREADS / 32], sf[NA_THREADS / 32];
    double rr = 0, ff = 0;
    const int64_t d0 = (int64_t)blockIdx.x * NA_PER_BLOCK;
    for (int64_t d = d0 + threadIdx.x; d < min(n_dof, d0 + NA_PER_BLOCK); d += NA_THREADS) {
        double fr = 0, fi = 0, rre = 0, rim = 0;
        for (int64_t p = copy_ptr[d]; p < copy_ptr[d + 1]; ++p) {
            const int64_t r = copy_idx[p];
            const int64_t sl = r >> 5;
            const int lane = (int)(r & 31);
            const int64_t base = slice_ptr[sl];
            const int w = (int)((slice_ptr[sl + 1] - base) >> 5);
            double ar = 0, ai = 0;
            for (int t = 0; t < w; ++t) {
                const int64_t idx = base + ((int64_t)t << 5) + lane;
                const double2 x = u[loc_gdof[col[idx]]];
                const double b = bvg ? bvg[idx] : 0.0;   // 3-D: + i B_Gamma u on the SELL pattern
                ar += val[idx] * x.x - b * x.y;
                ai += val[idx] * x.y + b * x.x;
            }
            const double2 xr = u[loc_gdof[r]];
            ar -= bg[r] * xr.y;                       // 2-D: + i B_Gamma u (diagonal impedance term)
            ai += bg[r] * xr.x;
            const double2 fl = f_loc[r];
            fr += fl.x; fi += fl.y;
            rre += fl.x - ar; rim += fl.y - ai;
        }
        rr += rre * rre + rim * rim;
        ff += fr * fr + fi * fi;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        ff += __shfl_down_sync(0xffffffffu, ff, o);
    }
    if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = rr; sf[threadIdx.x >> 5] = ff; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int q = 0; q < NA_THREADS / 32; ++q) { a += sr[q]; b += sf[q]; }
        scratch[blockIdx.x] = a;
        scratch[NA_MAX_BLOCKS + blockIdx.x] = b;
    }
}

// Sum the partials of the nb blocks (fixed order) into out = (||r||, ||f||).
__global__ void k_na_finish(int nb, const double* __restrict__ scratch, double* __restrict__ out) {
    __shared__ double sr[32], sf[32];
    double a = 0, b = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) { a += scratch[i]; b += scratch[NA_MAX_BLOCKS + i]; }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = a; sf[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { x += sr[q]; y += sf[q]; }
        out[0] = sqrt(x);
        out[1] = sqrt(y);
    }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached; the host-side name g_na_scratch is only a
// stand-in and must never be passed to a kernel.
static double* scratch_ptr() {
    static std::mutex mu;
    static double* ptrs[NA_MAX_DEVICES] = {};
    int dev = 0;
    THM_CUDA(cudaGetDevice(&dev));
    THM_REQUIRE(dev >= 0 && dev < NA_MAX_DEVICES, "device ordinal out of range for the no-allocation scratch");
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) fail(THM_ECUDA, std::string("cudaGetSymbolAddress(no-allocation scratch): ") +
                                                  cudaGetErrorString(e));
        ptrs[dev] = static_cast<double*>(p);
    }
    return ptrs[dev];
}

}  // namespace thm

using namespace thm;

extern "C" int thm_residual_noalloc(const thm_sys* s, const double* u, double* out) {
    try {
        if (!s || !u || !out) fail(THM_EINVAL, "NULL argument");
        const thm_mesh* m = s->m;
        const int64_t nb = (m->n_dof + NA_PER_BLOCK - 1) / NA_PER_BLOCK;
        if (nb > NA_MAX_BLOCKS)
            fail(THM_EINVAL, "thm_residual_noalloc: n_dof = " + std::to_string(m->n_dof) +
                                 " exceeds the no-allocation limit of " +
                                 std::to_string((int64_t)NA_MAX_BLOCKS * NA_PER_BLOCK) + " DOFs");
        double* scratch = scratch_ptr();
        if (nb > 0) {
            THM_LAUNCH(THM_K_DDM, s->st,
                       k_na_residual<<<(unsigned)nb, NA_THREADS, 0, s->st>>>(
                           m->n_dof, m->d_copy_ptr.p, m->d_copy_idx.p, m->d_loc_gdof.p, m->d_slice_ptr.p,
                           m->d_sell_col.p, s->kloc_val64(), s->bg64.p, m->dim == 3 ? s->bvg64.p : nullptr, s->f_res.p,
                           reinterpret_cast<const double2*>(u), scratch));
        }
        THM_LAUNCH(THM_K_DDM, s->st, k_na_finish<<<1, 256, 0, s->st>>>((int)nb, scratch, out));
        THM_CUDA(cudaGetLastError());
        return THM_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (...) {
        set_last_error("thm_residual_noalloc: unexpected host error");
        return THM_EINVAL;
    }
}

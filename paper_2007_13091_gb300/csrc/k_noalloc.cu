// Time-step reduction for callers that cannot allocate device memory.
//
// ugkwp_time_step_noalloc computes the time step of the step (convective
// spectral radii, Courant number C) from caller-owned device arrays, like the
// reduction inside ugkwp_step, but keeps its scratch -- one partial minimum per
// block of 256 cells -- in a file-scope __device__ array instead of a
// caller-provided workspace, so the call allocates nothing.  Built with
// --fmad=false: for the same W, volumes and projected areas the result equals
// the time step ugkwp_step uses, bit for bit.
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/ugkwp.h"

namespace {

constexpr int DT_BLOCK = 256;
constexpr int DT_MAX_BLOCKS = UGKWP_NOALLOC_MAX_CELLS / DT_BLOCK;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) double g_dt_partial[DT_MAX_BLOCKS];

__global__ void __launch_bounds__(DT_BLOCK) k_dt_partial(const double* __restrict__ W, const double* __restrict__ vol,
                                                         const double* __restrict__ dS, int nc, double R,
                                                         double* partial) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double r = __longlong_as_double(0x7ff0000000000000LL);
    if (i < nc) {
        const double rho = W[i];
        const double Ux = W[nc + i] / rho, Uy = W[2 * nc + i] / rho, Uz = W[3 * nc + i] / rho;
        const double U2 = (Ux * Ux + Uy * Uy) + Uz * Uz;
        const double pr = (W[4 * nc + i] - 0.5 * (rho * U2)) / 1.5;
        const double T = pr / (rho * R);
        if (rho > 0.0 && pr > 0.0 && isfinite(pr)) {
            const double c = 3.0 * sqrt(R * T);
            const double lam = ((fabs(Ux) + c) * dS[i] + (fabs(Uy) + c) * dS[nc + i]) + (fabs(Uz) + c) * dS[2 * nc + i];
            r = vol[i] / lam;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) r = fmin(r, __shfl_xor_sync(0xffffffffu, r, d));
    __shared__ double sh[DT_BLOCK / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < DT_BLOCK / 32 ? sh[threadIdx.x] : __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, d));
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024) k_dt_final(const double* __restrict__ partial, int nb, double CFL, double* dt) {
    double v = __longlong_as_double(0x7ff0000000000000LL);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) v = fmin(v, partial[j]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, d));
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) w = fmin(w, __shfl_xor_sync(0xffffffffu, w, d));
        if (threadIdx.x == 0) dt[0] = CFL * w;
    }
}

// Device address of g_dt_partial, looked up once per device (the host-side
// name of the array is only a stand-in for it) and kept for the life of the
// process: a device reset makes it stale (documented in the header).
std::mutex g_mu;
double* g_ptr[256] = {};

}  // namespace

namespace ugkwp {
// Stores the message returned by ugkwp_last_error (defined in api.cpp).
void set_last_error_message(const std::string& msg);
}

extern "C" int ugkwp_time_step_noalloc(const double* d_W, const double* d_vol, const double* d_dS, int32_t n_cells,
                                       double R, double CFL, double* d_dt, void* cuda_stream) {
    if (!d_W || !d_vol || !d_dS || !d_dt || n_cells <= 0 || !(R > 0.0) || !(CFL > 0.0 && CFL <= 1.0)) {
        ugkwp::set_last_error_message("ugkwp_time_step_noalloc: invalid argument");
        return UGKWP_E_ARG;
    }
    if (n_cells > UGKWP_NOALLOC_MAX_CELLS) {
        ugkwp::set_last_error_message("ugkwp_time_step_noalloc: n_cells exceeds UGKWP_NOALLOC_MAX_CELLS (" +
                                      std::to_string(UGKWP_NOALLOC_MAX_CELLS) + ")");
        return UGKWP_E_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        ugkwp::set_last_error_message(std::string("ugkwp_time_step_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return UGKWP_E_CUDA;
    }
    double* partial = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_ptr[dev]) {
            e = cudaGetSymbolAddress((void**)&g_ptr[dev], g_dt_partial);
            if (e != cudaSuccess) {
                g_ptr[dev] = nullptr;
                ugkwp::set_last_error_message(std::string("ugkwp_time_step_noalloc: cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e));
                return UGKWP_E_CUDA;
            }
        }
        partial = g_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nb = (n_cells + DT_BLOCK - 1) / DT_BLOCK;
    k_dt_partial<<<nb, DT_BLOCK, 0, st>>>(d_W, d_vol, d_dS, n_cells, R, partial);
    k_dt_final<<<1, 1024, 0, st>>>(partial, nb, CFL, d_dt);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        ugkwp::set_last_error_message(std::string("ugkwp_time_step_noalloc: launch: ") + cudaGetErrorString(e));
        return UGKWP_E_CUDA;
    }
    return UGKWP_OK;
}

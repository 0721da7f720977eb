// Allocation-free CFL time step (mhd_cfl_dt_uniform_noalloc, declared in
// include/mhd_bunch.h).
//
// Who needs it: callers that must not allocate device memory through the CUDA runtime --
// hosts whose framework owns every byte of device memory through its own pool (its
// allocator accounts for all memory, so a library that calls cudaMalloc behind it breaks
// that accounting), and real-time loops that cannot pay for an allocation.  The handle API
// (mhd_bunch_create) allocates its patch table and work buffers; this entry point needs no
// handle and allocates nothing.
//
// Its only scratch memory is the file-scope device array below (one partial maximum per
// patch plus a completion counter), so every GPU that loads the library keeps those
// 128 KB + 4 B until the process exits.  All calls share the array: calls whose kernels
// overlap on the GPU (e.g. on two streams at once) race on it and must be serialised by
// the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/mhd_bunch.h"
#include "mhd_common.cuh"
#include "mhd_launch.h"
#include "mhd_math.cuh"

namespace mhd {
void set_last_error(const std::string& msg);
}

using namespace mhd;

namespace {

constexpr int kMaxPatches = MHD_NOALLOC_MAX_PATCHES;
constexpr int kMaxDevices = 64;

// one partial maximum per patch (block) and the last-block counter
static __device__ __align__(256) double g_partial[kMaxPatches];
static __device__ __align__(256) unsigned g_counter;

// Device addresses of the array, looked up per device; a lookup that failed is not kept
// (the next call on that device tries again).
struct DevScratch {
    double* partial = nullptr;
    unsigned* counter = nullptr;
    bool ready = false;
};
DevScratch g_dev[kMaxDevices];
std::mutex g_dev_mutex;

int fail(int code, const std::string& msg) {
    set_last_error(msg);
    return code;
}

// Host code cannot use the address of a __device__ array directly (the name denotes a
// host-side stand-in); the real device address is looked up with the device current.
cudaError_t setup_device(int dev, DevScratch& out) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (!g_dev[dev].ready) {
        DevScratch s;
        cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.partial), g_partial);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.counter), g_counter);
        if (e != cudaSuccess) return e;
        s.ready = true;
        g_dev[dev] = s;
    }
    out = g_dev[dev];
    return cudaSuccess;
}

template <typename R>
__device__ __forceinline__ R wmax(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        R w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// One block per patch: the block's maximum of sum_d (|u_d| + c_f,d)/dx_d over the
// patch's interior cells goes to partial[p] (NaN when a cell's rate is not finite); the
// last block to finish reduces the partials and writes courant / max to *dt_out (NaN if
// any partial is NaN), then leaves the counter at zero.
template <typename R>
__global__ void cfl_uniform_kernel(const R* __restrict__ U, int npatch, int nx, int ny, int nz, int gx, int gy,
                                   int gz, double gamma_d, double courant, double dxi0_d, double dxi1_d,
                                   double dxi2_d, double* partial, unsigned* counter, double* dt_out) {
    __shared__ R red[32];
    __shared__ double redd[32];
    __shared__ int nbad;
    __shared__ bool last;
    if (threadIdx.x == 0) nbad = 0;
    __syncthreads();
    const int X = nx + 2 * gx, Y = ny + 2 * gy, Z = nz + 2 * gz;
    const int64_t vol = (int64_t)X * Y * Z;
    const int p = blockIdx.x;
    const R* base = U + (int64_t)p * 8 * vol;
    const R gamma = R(gamma_d), gm1 = R(gamma_d - 1.0);
    const R dxi0 = R(dxi0_d), dxi1 = R(dxi1_d), dxi2 = R(dxi2_d);
    const bool ay = ny > 1, az = nz > 1;
    R vmax = R(0);
    bool bad = false;
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const int64_t row = k / nx;
        const int x = (int)(k - row * nx) + gx, y = (int)(row % ny) + gy, z = (int)(row / ny) + gz;
        const R* c = base + ((int64_t)z * Y + y) * X + x;
        const R bxc = R(0.5) * (c[5 * vol] + c[5 * vol + 1]);
        const R byc = ay ? R(0.5) * (c[6 * vol] + c[6 * vol + X]) : c[6 * vol];
        const R bzc = az ? R(0.5) * (c[7 * vol] + c[7 * vol + (int64_t)X * Y]) : c[7 * vol];
        R q[8];
        cons_to_prim(c[0], c[vol], c[2 * vol], c[3 * vol], c[4 * vol], bxc, byc, bzc, gm1, q);
        const R ri = rdiv(R(1), q[Q_RHO]), gP = gamma * q[Q_P];
        R rate = (rabs(q[Q_U]) + fast_speed(ri, gP, bxc, byc, bzc)) * dxi0;
        if (ay) rate += (rabs(q[Q_V]) + fast_speed(ri, gP, byc, bzc, bxc)) * dxi1;
        if (az) rate += (rabs(q[Q_W]) + fast_speed(ri, gP, bzc, bxc, byc)) * dxi2;
        if (isfinite((double)rate)) vmax = rate > vmax ? rate : vmax;
        else bad = true;
    }
    if (bad) atomicAdd(&nbad, 1);
    vmax = wmax(vmax);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
    __syncthreads();
    if (threadIdx.x < 32) {
        R v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : R(0);
        v = wmax(v);
        if (threadIdx.x == 0) {
            partial[p] = nbad ? __longlong_as_double(0x7ff8000000000000ll) : (double)v;
            __threadfence();
            last = (atomicAdd(counter, 1u) == (unsigned)npatch - 1u);
        }
    }
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x == 0) nbad = 0;
        __syncthreads();
        double v = 0.0;
        bool anynan = false;
        for (int k = threadIdx.x; k < npatch; k += blockDim.x) {
            const double w = ((volatile double*)partial)[k];
            if (w != w) anynan = true;
            else v = w > v ? w : v;
        }
        if (anynan) atomicAdd(&nbad, 1);
        v = wmax(v);
        if ((threadIdx.x & 31) == 0) redd[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            double u = threadIdx.x < (blockDim.x >> 5) ? redd[threadIdx.x] : 0.0;
            u = wmax(u);
            if (threadIdx.x == 0) {
                *dt_out = nbad ? __longlong_as_double(0x7ff8000000000000ll) : courant / u;
                *counter = 0u;
            }
        }
    }
}

}  // namespace

extern "C" int mhd_cfl_dt_uniform_noalloc(const void* state, int real_bytes, int npatch, int nx, int ny, int nz,
                                          int guard, const double dx[3], double gamma, double courant,
                                          void* dt_dev, void* cuda_stream) try {
    if (!state || !dx || !dt_dev) return fail(MHD_EINVAL, "NULL argument");
    if (real_bytes != 4 && real_bytes != 8) return fail(MHD_EINVAL, "real_bytes must be 4 or 8");
    if (npatch <= 0) return fail(MHD_EINVAL, "npatch must be positive");
    if (npatch > kMaxPatches)
        return fail(MHD_EINVAL, "npatch exceeds MHD_NOALLOC_MAX_PATCHES (" + std::to_string(kMaxPatches) +
                                    "), the size of the static work array");
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096) return fail(MHD_EINVAL, "bad patch size");
    if ((nz > 1 && ny == 1) || nx == 1) return fail(MHD_EINVAL, "active axes must be x, x-y or x-y-z");
    if (guard < 3) return fail(MHD_EINVAL, "guard must be >= 3");
    for (int d = 0; d < 3; ++d)
        if (!(dx[d] > 0)) return fail(MHD_EINVAL, "dx must be positive");
    if (!(gamma > 1.0) || !(courant > 0.0)) return fail(MHD_EINVAL, "gamma must be > 1 and courant > 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(MHD_EINVAL, "device ordinal out of range");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int sdev = dev;
    e = cudaStreamGetDevice(st, &sdev);
    if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("cudaStreamGetDevice: ") + cudaGetErrorString(e));
    if (sdev != dev)
        return fail(MHD_EINVAL, "cuda_stream belongs to device " + std::to_string(sdev) + " but device " +
                                    std::to_string(dev) + " is current");
    DevScratch s;
    e = setup_device(dev, s);
    if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    // an error left pending on this thread by earlier, unrelated work is cleared here, so
    // that the check after the launch reports this call's own launch only
    (void)cudaGetLastError();
    e = cudaMemsetAsync(s.counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int gx = guard, gy = ny > 1 ? guard : 0, gz = nz > 1 ? guard : 0;
    const double dxi[3] = {1.0 / dx[0], 1.0 / dx[1], 1.0 / dx[2]};
    if (real_bytes == 4)
        cfl_uniform_kernel<float><<<npatch, 256, 0, st>>>(static_cast<const float*>(state), npatch, nx, ny, nz, gx,
                                                          gy, gz, gamma, courant, dxi[0], dxi[1], dxi[2], s.partial,
                                                          s.counter, static_cast<double*>(dt_dev));
    else
        cfl_uniform_kernel<double><<<npatch, 256, 0, st>>>(static_cast<const double*>(state), npatch, nx, ny, nz, gx,
                                                           gy, gz, gamma, courant, dxi[0], dxi[1], dxi[2], s.partial,
                                                           s.counter, static_cast<double*>(dt_dev));
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MHD_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return MHD_OK;
} MHD_CATCH_ALL

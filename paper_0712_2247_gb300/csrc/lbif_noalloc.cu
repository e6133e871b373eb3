// Profile reduction that allocates no memory, for callers that cannot.
//
// lbif_profiles() reduces a handle's fields through a buffer the handle
// allocated. Some callers cannot allocate device memory at the moment they
// need profiles: services that reserved their whole device budget up front
// through their own allocator (a further cudaMalloc would fail or fragment
// it), or real-time loops that must keep a fixed memory footprint. This entry
// point works on density and velocity fields the caller already holds (for
// example tensors filled by lbif_moments with on_device = 1) and keeps its
// only intermediate, the per-plane sums, in a fixed-size array in the
// library's device image.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "lbif.h"

namespace {

constexpr int kMaxPlanes = 8192;          // largest nz accepted
constexpr int kMaxDevices = 64;
constexpr int kSlots = 5 * kMaxPlanes + 4;  // 5 per-plane sums, then 4 totals

// Every GPU that loads the library holds these 320 KB until the process exits.
// All calls share it: calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_sums[kSlots];

// Host-side device addresses of g_sums, one per device, looked up at the first
// call on the device and again whenever the device's current context changed
// since (a reset device reloads the library's image at a new address).
struct SumsAddr {
    CUcontext ctx;
    double* ptr;
};
static SumsAddr g_addr[kMaxDevices];
static std::mutex g_addr_lock;

// cuCtxGetCurrent through the runtime's driver entry point (no link against
// the driver library); NULL if unavailable
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
static CtxGetCurrentFn ctx_get_current()
{
    static std::once_flag once;
    static CtxGetCurrentFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// per plane z: sum rho, sum u_x, sum rho u_x, sum rho u_y, sum rho u_z (FP64,
// fixed-order tree); slot k of plane z at sums[k * kMaxPlanes + z]
__global__ void k_plane_sums(const float* __restrict__ rho, const float* __restrict__ u, int nx, int ny,
                             long long N, double* sums)
{
    __shared__ double sh[5][256];
    const int z = blockIdx.x;
    const long long A = (long long)nx * ny;
    double a[5] = {0, 0, 0, 0, 0};
    for (long long k = threadIdx.x; k < A; k += blockDim.x) {
        const long long i = (long long)z * A + k;
        const double r = rho[i], vx = u[i], vy = u[N + i], vz = u[2 * N + i];
        a[0] += r;
        a[1] += vx;
        a[2] += r * vx;
        a[3] += r * vy;
        a[4] += r * vz;
    }
    for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] = a[j];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 5) sums[(long long)threadIdx.x * kMaxPlanes + z] = sh[threadIdx.x][0];
}

// totals over planes (fixed order): mass, momentum x, y, z
__global__ void k_totals(int nz, double* sums)
{
    if (threadIdx.x >= 4) return;
    const int slot = threadIdx.x == 0 ? 0 : threadIdx.x + 1;
    double t = 0.0;
    for (int z = 0; z < nz; ++z) t += sums[(long long)slot * kMaxPlanes + z];
    sums[5 * kMaxPlanes + threadIdx.x] = t;
}

int device_sums(double** out, std::string& err)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return LBIF_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device index out of range";
        return LBIF_ERR_UNSUPPORTED;
    }
    // make the device's primary context current (initialised if it was not;
    // nothing is allocated), so that the context read below is the one the
    // launches will use
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return LBIF_ERR_CUDA;
    }
    CUcontext ctx = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    std::lock_guard<std::mutex> lock(g_addr_lock);
    SumsAddr& a = g_addr[dev];
    if (!a.ptr || a.ctx != ctx) {
        // set-up once per device (and context), with that device current
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_sums);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return LBIF_ERR_CUDA;
        }
        a.ptr = p;
        a.ctx = ctx;
    }
    *out = a.ptr;
    return LBIF_OK;
}

thread_local std::string g_msg = "no error";

}  // namespace

extern "C" const char* lbif_noalloc_last_error(void) { return g_msg.c_str(); }

extern "C" int lbif_field_profiles_noalloc(const float* rho, const float* u, int32_t nx, int32_t ny,
                                           int32_t nz, double* n_z, double* ux_z, double* out4,
                                           void* stream)
{
    if (!rho || !u || nx < 1 || ny < 1 || nz < 1) {
        g_msg = "lbif_field_profiles_noalloc: bad arguments";
        return LBIF_ERR_ARG;
    }
    if (nz > kMaxPlanes) {
        g_msg = "lbif_field_profiles_noalloc: nz = " + std::to_string(nz) + " exceeds the fixed limit of " +
                std::to_string(kMaxPlanes) + " planes";
        return LBIF_ERR_UNSUPPORTED;
    }
    double* sums = nullptr;
    int rc = device_sums(&sums, g_msg);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = (long long)nx * ny * nz;
    k_plane_sums<<<nz, 256, 0, s>>>(rho, u, nx, ny, N, sums);
    k_totals<<<1, 32, 0, s>>>(nz, sums);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && n_z) e = cudaMemcpyAsync(n_z, sums, sizeof(double) * nz, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && ux_z)
        e = cudaMemcpyAsync(ux_z, sums + kMaxPlanes, sizeof(double) * nz, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && out4)
        e = cudaMemcpyAsync(out4, sums + 5 * kMaxPlanes, sizeof(double) * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        g_msg = std::string("lbif_field_profiles_noalloc: ") + cudaGetErrorString(e);
        return LBIF_ERR_CUDA;
    }
    const double A = (double)nx * ny;
    for (int z = 0; z < nz; ++z) {
        if (n_z) n_z[z] /= A;
        if (ux_z) ux_z[z] /= A;
    }
    return LBIF_OK;
}

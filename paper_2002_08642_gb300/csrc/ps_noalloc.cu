// ps_noalloc.cu -- penalization force and moment of caller-supplied fields
// without any device allocation.
//
// Who needs this: callers that must not call cudaMalloc after start-up.
// Examples:
//   * a real-time control loop: cudaMalloc can block and synchronise the
//     device;
//   * a process whose framework's memory pool already holds nearly all
//     device memory, where a fresh cudaMalloc fails;
//   * code under a no-dynamic-allocation rule.
// Such callers cannot create a ps_ctx, whose workspace is gigabytes of
// caller memory, just to reduce a force. This entry point keeps its only
// scratch, one partial sum per x-plane, in a fixed array compiled into the
// library.
//
// The scratch: ps_noalloc_partials, 1024 planes x 6 doubles (48 KiB) per
// device that loads the library, held until the process exits. Grids with
// n > 1024 are rejected (PS_EINVAL). Each call writes every partial it later
// reads, so nothing carries over between calls. But all calls share the
// array: two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race, and must not be issued.
//
// Device-address set-up: host code cannot pass the array's name to a kernel
// (on the host it is only a stand-in symbol). So the first call on each
// device, with that device current, looks the address up with
// cudaGetSymbolAddress and caches it per device number. The cached address
// belongs to the device's current context: after cudaDeviceReset it is
// stale, and the call must not be used again in that process.
//
// It makes CUDA runtime calls (launches, error queries), so it must not be
// called from a stream callback or a host function queued with
// cudaLaunchHostFunc: CUDA forbids CUDA calls there.
#include <mutex>

#include "ps.h"
#include "ps_kernels.cuh"

static constexpr int kNoallocMaxPlanes = 1024;
static constexpr int kNoallocMaxDevices = 64;

// The fixed scratch: one 6-double partial sum per x-plane.
static __device__ __align__(256) double ps_noalloc_partials[kNoallocMaxPlanes * 6];

namespace {

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoallocMaxDevices] = {};

// One block per x-plane: chi (u - u_s) and (x - x0) x chi (u - u_s) summed
// in double (Neumaier per thread, then a block tree) into the plane's slot.
template <typename T>
__global__ void k_force_planes(int n, double dx, double x0, double y0, double z0, const T* __restrict__ u,
                               const T* __restrict__ chi, const T* __restrict__ us, double* __restrict__ part) {
    __shared__ double red[32 * 6];
    const int ix = blockIdx.x;
    const size_t n2 = (size_t)n * n, n3 = n2 * n, base = (size_t)ix * n2;
    ps::Acc acc[6] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (size_t i = threadIdx.x; i < n2; i += blockDim.x) {
        const size_t p = base + i;
        const double c = (double)chi[p];
        if (c == 0.0) continue;
        const int iy = (int)(i / n), iz = (int)(i % n);
        const double px = c * ((double)u[p] - (double)us[p]);
        const double py = c * ((double)u[n3 + p] - (double)us[n3 + p]);
        const double pz = c * ((double)u[2 * n3 + p] - (double)us[2 * n3 + p]);
        const double rx = ix * dx - x0, ry = iy * dx - y0, rz = iz * dx - z0;
        acc[0].add(px);
        acc[1].add(py);
        acc[2].add(pz);
        acc[3].add(ry * pz - rz * py);
        acc[4].add(rz * px - rx * pz);
        acc[5].add(rx * py - ry * px);
    }
    double v[6];
    for (int k = 0; k < 6; ++k) v[k] = acc[k].val();
    ps::block_sum<6>(v, part + (size_t)ix * 6, red);
}

// Planes summed in index order (Neumaier), scaled by dx^3 / eta.
__global__ void k_force_planes_final(int n, double scale, const double* __restrict__ part, double* __restrict__ FM) {
    if (threadIdx.x >= 6) return;
    ps::Acc a = {0, 0};
    for (int ix = 0; ix < n; ++ix) a.add(part[(size_t)ix * 6 + threadIdx.x]);
    FM[threadIdx.x] = a.val() * scale;
}

}  // namespace

extern "C" ps_status ps_penalization_force_noalloc(int32_t n, int32_t precision, double L, double eta,
                                                   const double x0[3], const void* u_dev, const void* chi_dev,
                                                   const void* us_dev, double* FM_dev, void* cuda_stream) {
    if (n < 1 || n > kNoallocMaxPlanes) return PS_EINVAL;
    if (precision != PS_FP32 && precision != PS_FP64) return PS_EINVAL;
    if (!(L > 0) || !(eta > 0) || !x0 || !u_dev || !chi_dev || !us_dev || !FM_dev) return PS_EINVAL;
    // an error left by earlier work on this thread stays in place for the
    // code that caused it; this call does not start on top of it
    if (cudaPeekAtLastError() != cudaSuccess) return PS_ECUDA;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return PS_ECUDA;
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, ps_noalloc_partials) != cudaSuccess || !p) return PS_ECUDA;
            g_noalloc_ptr[dev] = (double*)p;
        }
        part = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const double dx = L / n;
    // each launch checked on its own (a failed launch's error is this call's)
    if (precision == PS_FP64)
        k_force_planes<double><<<n, 256, 0, s>>>(n, dx, x0[0], x0[1], x0[2], (const double*)u_dev,
                                                 (const double*)chi_dev, (const double*)us_dev, part);
    else
        k_force_planes<float><<<n, 256, 0, s>>>(n, dx, x0[0], x0[1], x0[2], (const float*)u_dev,
                                                (const float*)chi_dev, (const float*)us_dev, part);
    if (cudaGetLastError() != cudaSuccess) return PS_ECUDA;
    k_force_planes_final<<<1, 32, 0, s>>>(n, dx * dx * dx / eta, part, FM_dev);
    if (cudaGetLastError() != cudaSuccess) return PS_ECUDA;
    return PS_OK;
}

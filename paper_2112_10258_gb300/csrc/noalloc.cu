// sift3d_gaussian_blur_noalloc: the separable 3D Gaussian blur for callers that
// cannot allocate device memory themselves - code running where cudaMalloc is
// unavailable or forbidden (a custom allocator's own reclaim path, a real-time
// loop that must not touch the allocator, or an embedding that hands the
// library only its input and output buffers).  It makes CUDA calls (kernel
// launches; a symbol lookup on the first call per device), so it cannot run
// inside a host function or callback enqueued on a stream.
//
// The two float32 intermediate volumes live in one file-scope device array that
// every GPU which loads this library holds until the process exits.  Host code
// cannot pass the array's name to a kernel (on the host it is only a stand-in
// symbol), so each device's address is obtained once with cudaGetSymbolAddress
// while that device is current, and the kernels receive that address.
#include <mutex>

#include "runtime.hpp"

namespace {

constexpr int64_t kNoallocElems = SIFT3D_BLUR_NOALLOC_MAX_ELEMS;   // per intermediate volume

// T (after the y and x passes) and U (after the z pass), back to back.
static __device__ __align__(256) float g_blur_scratch[2 * kNoallocElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" int sift3d_gaussian_blur_noalloc(const float* dev_in, int nx, int ny, int nz, double sigma, double trunc,
                                            float* dev_out, void* stream) {
    if (!dev_in || !dev_out) return SIFT3D_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4095 || ny > 4095 || nz > 4095) return SIFT3D_EINVAL;
    if (!(trunc > 0.0) || !(trunc <= 10.0)) return SIFT3D_EINVAL;
    const int R = sift3d::gaussian_radius(sigma, trunc);
    if (!(sigma > 0.0) || R < 1 || R > sift3d::kMaxRadius) return SIFT3D_EINVAL;
    // The rows of each intermediate are padded to a multiple of 8 floats.
    if (sift3d::blur_pitch_elems(nx, ny, nz) > kNoallocElems) return SIFT3D_ECAPACITY;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SIFT3D_ECUDA;
    float* base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (g_scratch_addr[dev] == nullptr) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_blur_scratch) != cudaSuccess || p == nullptr) {
                (void)cudaGetLastError();
                return SIFT3D_ECUDA;
            }
            g_scratch_addr[dev] = static_cast<float*>(p);
        }
        base = g_scratch_addr[dev];
    }
    // Every intermediate element is written before it is read, so the array's
    // contents from an earlier call need no clearing.
    return sift3d::enqueue_blur(dev_in, nx, ny, nz, sigma, trunc, base, base + kNoallocElems, dev_out,
                                static_cast<cudaStream_t>(stream), nullptr);
}

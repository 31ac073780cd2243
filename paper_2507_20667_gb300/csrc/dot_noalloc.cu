// Inner product of two device vectors with FP64 accumulation that allocates no memory.
//
// Some callers cannot allocate device memory while they run: code whose device memory is handed
// out by a host framework's own pool (which then owns the whole device and forbids side
// allocations), latency-critical serving loops where cudaMalloc / cudaFree would stall every
// stream on the device (both synchronize implicitly) or could fail under memory pressure in the
// middle of a request.  For them this file keeps its scratch -- one FP64 partial sum per block --
// in a file-scope device array that every GPU loading the library holds until the process exits.
//
// The computation is the final-reduction kernel class of the engine (the scalar-producing root
// step, products in the storage precision summed in runs of 32 and then in FP64), here on two
// caller-owned vectors of the same layout.
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "tnsa.h"
#include "tn_internal.hpp"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kChunk = 65536;             // elements reduced by one block
constexpr int kMaxBlocks = 1024;              // capacity of the scratch array
constexpr int64_t kMaxElems = kChunk * kMaxBlocks;   // 2^26 elements per call
constexpr int kMaxDevices = 64;

// The scratch: one partial sum per block of the first kernel.  Every call overwrites the entries
// it uses before reading them, so nothing has to start at zero.
static __device__ __align__(256) double2 g_dot_scratch[kMaxBlocks];

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot_chunks(const typename Cx<T>::t *__restrict__ a,
                                                         const typename Cx<T>::t *__restrict__ b,
                                                         int64_t n, double2 *__restrict__ partials) {
    __shared__ double2 red[kThreads / 32];
    const int64_t begin = (int64_t)blockIdx.x * kChunk;
    const int64_t end = begin + kChunk < n ? begin + kChunk : n;
    double sx = 0, sy = 0;
    T rx = 0, ry = 0;
    int cnt = 0;
    for (int64_t i = begin + threadIdx.x; i < end; i += kThreads) {
        const typename Cx<T>::t x = a[i], y = b[i];
        rx = fma(x.x, y.x, rx);
        rx = fma(-x.y, y.y, rx);
        ry = fma(x.x, y.y, ry);
        ry = fma(x.y, y.x, ry);
        if (++cnt == 32) {
            sx += (double)rx;
            sy += (double)ry;
            rx = ry = 0;
            cnt = 0;
        }
    }
    sx += (double)rx;
    sy += (double)ry;
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(sx, sy);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = make_double2(0, 0);
        for (int w = 0; w < kThreads / 32; ++w) { s.x += red[w].x; s.y += red[w].y; }
        partials[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads) k_dot_sum(const double2 *__restrict__ partials, int32_t nblocks,
                                                      double *__restrict__ out) {
    __shared__ double2 red[kThreads / 32];
    double sx = 0, sy = 0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) {
        sx += partials[i].x;
        sy += partials[i].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(sx, sy);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = make_double2(0, 0);
        for (int w = 0; w < kThreads / 32; ++w) { s.x += red[w].x; s.y += red[w].y; }
        out[0] = s.x;
        out[1] = s.y;
    }
}

// Device address of the scratch array, looked up once per device with that device current.  The
// address belongs to the device's primary context as it was at the lookup: a cudaDeviceReset
// destroys that context (the module is loaded again by the next call and the array may move), so
// a caller that resets a device must not call tn_dot_noalloc on it afterwards.
std::mutex g_mu;
double2 *g_scratch_ptr[kMaxDevices] = {};

tn_status scratch_for(int32_t device, double2 **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dot_scratch);
        if (e != cudaSuccess)
            return tn::fail(TN_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[device] = static_cast<double2 *>(p);
    }
    *out = g_scratch_ptr[device];
    return TN_OK;
}

}  // namespace

extern "C" tn_status tn_dot_noalloc(int32_t device, void *cuda_stream, const void *d_a,
                                    const void *d_b, int64_t n, tn_precision prec, double *d_out) {
    if (!d_out || (n > 0 && (!d_a || !d_b))) return tn::fail(TN_EINVAL, "NULL argument");
    if (n < 0) return tn::fail(TN_EINVAL, "n must be >= 0");
    if (n > kMaxElems)
        return tn::fail(TN_EINVAL, "n = " + std::to_string(n) + " exceeds the no-allocation limit of " +
                                       std::to_string(kMaxElems) + " elements (2^26)");
    if (prec != TN_C64 && prec != TN_C128)
        return tn::fail(TN_EINVAL, "tn_dot_noalloc takes TN_C64 or TN_C128 vectors");
    if (device < 0 || device >= kMaxDevices) return tn::fail(TN_EINVAL, "device index out of range");
    // the call works on `device` and leaves the caller's current device as it found it
    int caller_device = -1;
    cudaError_t e = cudaGetDevice(&caller_device);
    if (e != cudaSuccess) return tn::fail(TN_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    struct Restore {
        int dev, cur;
        ~Restore() { if (dev != cur) cudaSetDevice(dev); }
    } restore{caller_device, device};
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return tn::fail(TN_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    double2 *scratch = nullptr;
    tn_status s = scratch_for(device, &scratch);
    if (s != TN_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int32_t blocks = (int32_t)((n + kChunk - 1) / kChunk);
    if (blocks > 0) {
        if (prec == TN_C64)
            k_dot_chunks<float><<<blocks, kThreads, 0, st>>>(static_cast<const float2 *>(d_a),
                                                             static_cast<const float2 *>(d_b), n, scratch);
        else
            k_dot_chunks<double><<<blocks, kThreads, 0, st>>>(static_cast<const double2 *>(d_a),
                                                              static_cast<const double2 *>(d_b), n, scratch);
    }
    k_dot_sum<<<1, kThreads, 0, st>>>(scratch, blocks, d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return tn::fail(TN_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return TN_OK;
}

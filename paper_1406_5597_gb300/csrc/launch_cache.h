// Launch set-up that belongs to a device.  A kernel's dynamic shared memory
// limit, and the occupancy figures derived from it, are properties of the
// device's context, so launchers keep them per device ordinal rather than
// per process.  The cache cells are atomics: concurrent first launches from
// several host threads may both run the set-up, which gives the same value.
#pragma once
#include <atomic>

#include <cuda_runtime.h>

namespace fft3d {

constexpr int kMaxCachedDevices = 64;

// One positive int per device; 0 = not set up yet on that device.
struct PerDevice {
    std::atomic<int> v[kMaxCachedDevices] = {};
};

// The cached value of the current device, computed on first use by
// setup(dev, &value) (a cudaError_t; value must come out >= 1).  Devices
// beyond the table run the set-up on every call.
template <class F>
inline cudaError_t per_device(PerDevice& c, int* out, F&& setup)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < kMaxCachedDevices;
    if (cached) {
        const int v = c.v[dev].load(std::memory_order_acquire);
        if (v > 0) {
            *out = v;
            return cudaSuccess;
        }
    }
    int v = 0;
    e = setup(dev, &v);
    if (e != cudaSuccess) return e;
    if (v < 1) return cudaErrorInvalidConfiguration;
    if (cached) c.v[dev].store(v, std::memory_order_release);
    *out = v;
    return cudaSuccess;
}

// Raise kernel k's dynamic shared memory limit to smem, once per device.
template <class K>
inline cudaError_t smem_limit_per_device(PerDevice& c, K k, size_t smem)
{
    int done = 0;
    return per_device(c, &done, [&](int, int* v) {
        *v = 1;
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
}

// Resident CTAs of kernel k on the whole current device (CTAs per SM times
// SMs) with `threads` threads and smem bytes of dynamic shared memory; sets
// the shared memory limit first.  Once per device.
template <class K>
inline cudaError_t resident_ctas_per_device(PerDevice& c, K k, int threads, size_t smem, int* out)
{
    return per_device(c, out, [&](int dev, int* v) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
        if (e != cudaSuccess) return e;
        *v = per_sm * sms;
        return cudaSuccess;
    });
}

}  // namespace fft3d

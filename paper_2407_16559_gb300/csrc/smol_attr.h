// smol_attr.h - host-side kernel attributes shared by every entry point of the library.
//
// cudaFuncAttributeMaxDynamicSharedMemorySize is one setting per kernel and device,
// shared by every system, batch and standalone call that launches that kernel. A call
// that set it to its own (smaller) need would make a launch of a larger live system
// fail, so the limit only ever rises: raise_smem keeps a high-water mark per (kernel,
// device) under a mutex and calls cudaFuncSetAttribute only to raise it.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

namespace smol_host {

inline std::mutex& smem_mutex() {
    static std::mutex m;
    return m;
}
inline std::map<std::pair<const void*, int>, int>& smem_marks() {
    static std::map<std::pair<const void*, int>, int> m;
    return m;
}

// Makes kernel k accept at least `bytes` of dynamic shared memory on the current device;
// never lowers a limit set before (by this or any other caller in the process).
template <typename K>
cudaError_t raise_smem(K k, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(smem_mutex());
    const std::pair<const void*, int> key((const void*)k, dev);
    auto it = smem_marks().find(key);
    if (it != smem_marks().end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) smem_marks()[key] = bytes;
    return e;
}

}  // namespace smol_host

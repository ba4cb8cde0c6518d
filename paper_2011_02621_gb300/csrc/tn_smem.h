// Per-device kernel attributes shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#define TN_MAX_DEVICES 64

// Raise a kernel's dynamic shared memory limit to the most the current device allows next to the
// kernel's static shared memory. The attribute belongs to the device's context, so it is set once
// per device: the table is per kernel (the kernel is the template argument, so two kernels of the
// same signature keep separate tables) and indexed by the device ordinal. Later launches on that
// device ask for at most the limit. Returns the limit in bytes, or -1 when a CUDA call failed.
template <auto Kernel>
inline int tn_smem_optin() {
  static int limit[TN_MAX_DEVICES];   // 0 = not yet set on that device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TN_MAX_DEVICES) return -1;
  int lim = __atomic_load_n(&limit[dev], __ATOMIC_ACQUIRE);
  if (lim != 0) return lim;
  int optin = 0;
  cudaFuncAttributes fa;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, Kernel) != cudaSuccess)
    return -1;
  lim = optin - (int)fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) return -1;
  __atomic_store_n(&limit[dev], lim, __ATOMIC_RELEASE);
  return lim;
}

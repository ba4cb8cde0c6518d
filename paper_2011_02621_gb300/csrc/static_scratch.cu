// tn_amplitudes_static: tn_amplitudes without any device allocation.
//
// Some callers cannot let a library allocate device memory while they run: processes whose own
// memory pool has reserved the GPU's memory up front and accounts for every byte (a further
// cudaMalloc would fail or break that accounting), real-time or embedded hosts that may only use
// a fixed budget decided at start-up, and code that runs inside an allocator callback, where
// allocating again would re-enter that allocator. For them this entry point runs the same
// computation as tn_amplitudes, with every scratch buffer (bitstrings, bra tensors, SVD work,
// intermediates, overlap tensors, results, error words) carved out of one statically sized
// device array that lives in this file. Each GPU that loads the library holds that array
// (TN_STATIC_SCRATCH_BYTES) until the process exits.
#include <algorithm>
#include <mutex>

#include "tn_host.h"

#define TN_STATIC_SCRATCH_BYTES (size_t(32) << 20)   // 32 MiB per device

static __device__ __align__(256) unsigned char tn_static_scratch[TN_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_scratch_mu;
void *g_scratch_addr[256] = {};

// The array's device address on the current device. In host code the array's name is only a
// stand-in, so the address is asked once per device (with that device current) and cached.
tn_status scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tn_fail(TN_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return tn_fail(TN_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, tn_static_scratch);
    if (e != cudaSuccess || !p)
      return tn_fail(TN_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return TN_OK;
}

}  // namespace

extern "C" tn_status tn_amplitudes_static(tn_plan *p, const uint64_t *bits, int64_t n, tn_precision prec,
                                          tn_c128 *out, void *cuda_stream) {
  if (!p) return tn_fail(TN_ERR_ARG, "tn_amplitudes_static: NULL plan");
  if (prec < TN_FP64 || prec > TN_TF32X6) return tn_fail(TN_ERR_ARG, "unknown precision %d", (int)prec);
  if (n == 0) return TN_OK;
  if (n < 0 || !bits || !out) return tn_fail(TN_ERR_ARG, "tn_amplitudes_static: bad arguments");
  const int kind = prec == TN_FP64 ? 0 : 1;
  const int64_t cap = (int64_t)TN_STATIC_SCRATCH_BYTES;
  // as many whole bitstrings as fit; else one bitstring with as many of its slices as fit
  int64_t ch = 0, sc = p->n_slices;
  {
    const int64_t one = ws_sizes(p, kind, 1, sc).total;
    if (one <= cap) {
      ch = cap / one;
      ch = std::min<int64_t>(std::min<int64_t>(ch, n), 1 << 16);
      while (ch > 1 && ws_sizes(p, kind, ch, sc).total > cap) --ch;
    } else {
      ch = 1;
      while (sc > 1 && ws_sizes(p, kind, 1, sc).total > cap) sc = (sc + 1) / 2;
      if (ws_sizes(p, kind, 1, sc).total > cap)
        return tn_fail(TN_ERR_UNSUPPORTED,
                       "tn_amplitudes_static: one bitstring and one slice need %lld bytes of scratch, more than the "
                       "%lld-byte static scratch; use tn_amplitudes or more cuts (smaller max_intermediate)",
                       (long long)ws_sizes(p, kind, 1, 1).total, (long long)cap);
    }
  }
  // the array belongs to the device that is current; the plan's tensors live on its circuit's device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tn_fail(TN_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev != p->c->device)
    return tn_fail(TN_ERR_ARG, "tn_amplitudes_static: device %d is current, the plan lives on device %d", dev,
                   p->c->device);
  void *base = nullptr;
  tn_status s = scratch_address(&base);
  if (s != TN_OK) return s;
  // a workspace carved from the static array: run in its batch size, never grown or released
  Workspace w;
  ws_carve(w, base, ws_sizes(p, kind, ch, sc), ch, sc, (cudaStream_t)cuda_stream);
  w.fixed = true;
  // the error words are cleared by the run itself; every other buffer is written before read
  return run_amplitudes(p, w, bits, n, prec, out, (cudaStream_t)cuda_stream);
}

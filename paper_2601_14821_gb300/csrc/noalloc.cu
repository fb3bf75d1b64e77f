// noalloc.cu -- potr_bin_sort_static: the binning + radix sort of potr_bin_sort for callers
// that cannot allocate device memory, with its scratch in a fixed array of this library.
//
// Who needs it: code that runs inside a host application which owns every device
// allocation (a renderer or engine plug-in handed only its input and output buffers), code
// on a path where an allocation would synchronise the device or is forbidden (a latency-
// critical serving loop, an allocator-free embedded build), and callers that simply have no
// allocator bound to the device at that point.  Such callers still provide their inputs and
// outputs; the sort's scratch (scan partials, key/value double buffers, digit histograms)
// comes from g_bin_sort_scratch below.
//
// The array is a file-scope __device__ variable: every GPU that loads this library holds
// its kStaticScratchBytes until the process exits.  Its host-side name is only a stand-in
// for the symbol, not a device address, so the device address is looked up with
// cudaGetSymbolAddress (with that device current) on every call made outside a stream capture
// -- a context that was reset or replaced gets the array's new address -- and cached per device
// for calls made while their stream is being captured.  The first call on a device must come
// before any capture (a first call inside a capture is refused with POTR_ERR_UNSUPPORTED).
// All calls share the one array and it keeps the previous call's contents: nothing in it
// needs to start at zero (every word is written before it is read within a call), and calls
// whose work overlaps on the GPU race on it -- serialise them (one stream, or events).
#include <mutex>

#include "potr_device.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(56) << 20;  // 56 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bin_sort_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_bin_sort_scratch on the current device: looked up afresh outside a
// stream capture, the cached address inside one.
potr_status scratch_for_current_device(cudaStream_t s, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return POTR_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return POTR_ERR_UNSUPPORTED;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return POTR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bin_sort_scratch) != cudaSuccess || p == nullptr) return POTR_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  } else if (!g_scratch_ptr[dev]) {
    return POTR_ERR_UNSUPPORTED;  // the first call on a device came inside a capture
  }
  *out = g_scratch_ptr[dev];
  return POTR_OK;
}

}  // namespace

extern "C" potr_status potr_bin_sort_static(const potr_views* views, const potr_frame* frame,
                                            const potr_raster_config* cfg, int64_t n, int64_t instance_capacity,
                                            uint32_t* d_tiles, uint32_t* d_vals, uint32_t* d_tile_ranges,
                                            potr_device_status* d_status, potr_stream_t stream) {
  if (!views || !frame || !cfg || n <= 0 || frame->n_views < 1 || instance_capacity <= 0)
    return POTR_ERR_INVALID_ARGUMENT;
  if (instance_capacity > POTR_STATIC_MAX_INSTANCES) return POTR_ERR_TOO_LARGE;
  if (n * (int64_t)frame->n_views > POTR_STATIC_MAX_VIEW_SPLATS) return POTR_ERR_TOO_LARGE;
  const size_t need = potr_bin_sort_workspace_size(n, frame->n_views, frame->total_tiles, instance_capacity);
  if (need == 0) return POTR_ERR_INVALID_ARGUMENT;
  if (need > kStaticScratchBytes) return POTR_ERR_TOO_LARGE;
  void* scratch = nullptr;
  const potr_status st = scratch_for_current_device(reinterpret_cast<cudaStream_t>(stream), &scratch);
  if (st != POTR_OK) return st;
  return potr_bin_sort(views, frame, cfg, n, instance_capacity, d_tiles, d_vals, d_tile_ranges, d_status, scratch,
                       kStaticScratchBytes, stream);
}

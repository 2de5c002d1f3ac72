// interp_compress_noalloc: compression for callers that cannot allocate
// device memory themselves.
//
// Some callers have no way to provide the scratch buffer interp_compress
// needs: their device memory belongs to another allocator that they cannot
// ask for more (a host application's memory pool), they run in a plug-in
// host that forbids device allocation, or they are latency-critical loops
// that must never pay for a cudaMalloc and the synchronisation it implies.
// This entry point uses a scratch array compiled into the library instead.
//
// The array is a file-scope __device__ variable of kNoAllocScratchBytes
// (24 MiB): every GPU on which the library's code is loaded holds it until
// the process exits.  Host code cannot use the array's name as a device
// address (on the host it names a stand-in object), so every call made outside
// stream capture, with the device current, looks up the array's device address
// with cudaGetSymbolAddress (a device reset may move the array) and keeps it
// for that device; a call during capture uses the kept address, so one call on
// the device must come before any capture.  All calls share the one array:
// compression clears the parts that must start at zero (control words and
// outlier block counters) at the start of every call, and two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on the array and corrupt each other's results.
#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(24) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void *g_scratch_addr[kMaxDevices];  // device address of the array, per device (null until looked up)

}  // namespace

extern "C" size_t interp_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

extern "C" int interp_compress_noalloc(const float *d_x, const int64_t dims[3], double eb, const interp_config *cfg,
                                       float *d_anchors, uint16_t *d_codes, uint32_t *d_out_idx, float *d_out_val,
                                       uint64_t out_capacity, uint32_t *d_hist, interp_header *d_hdr,
                                       interp_stream_t stream)
{
    const size_t need = interp_workspace_bytes(dims, cfg);
    if (need == 0) return INTERP_EINVAL;
    if (need > kNoAllocScratchBytes) return INTERP_ESCRATCH;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return INTERP_ECUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cap) != cudaSuccess) return INTERP_ECUDA;
    if (cap == cudaStreamCaptureStatusNone) {
        // outside capture: look the address up every time (a device reset may move the array)
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return INTERP_ECUDA;
        g_scratch_addr[dev] = p;
    } else if (!g_scratch_addr[dev]) {
        return INTERP_ECUDA;  // captured before any call on this device looked the address up
    }
    return interp_compress(d_x, dims, eb, cfg, d_anchors, d_codes, d_out_idx, d_out_val, out_capacity, d_hist,
                           d_hdr, g_scratch_addr[dev], kNoAllocScratchBytes, stream);
}

// noalloc.cu -- corner detection for callers that cannot allocate device memory.
//
// Some callers own no device allocations of their own: a plugin inside a host
// application whose device memory belongs to that application's pool (raw
// cudaMalloc is not allowed there), or a real-time loop that must never call
// cudaMalloc / cudaFree, which can synchronise the device and break the frame
// cadence.  stab_detect_noalloc serves them: it runs the same detection kernels
// as stab_detect (response + NMS, histogram cut, exact top-K), but every piece
// of scratch they need -- the stream descriptor, its counters, the score
// histogram and the candidate keys -- lives in one file-scope device array of
// fixed size, so the call allocates nothing.  The caller still passes the
// frame and the output buffers.
//
// Limits: the ROI may be at most 1536 x 864 pixels (the reduced region of
// interest of a 1920 x 1080 frame) and max_corners at most 2048; the array is
// about 5.4 MB, held by every GPU that loads the library until the process
// exits.  Larger requests are rejected with STAB_ERR_CAPACITY.
#include <cstdio>
#include <mutex>

#include "kernels.cuh"

namespace {

constexpr int kMaxRoiW = 1536, kMaxRoiH = 864;
constexpr long long kCap = (long long)((kMaxRoiW + 1) / 2) * ((kMaxRoiH + 1) / 2) + 64;   // NMS survivors
constexpr size_t kAlign = 256;
constexpr size_t al(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffDesc = 0;
constexpr size_t kOffState = al(kOffDesc + sizeof(StreamDev));
constexpr size_t kOffPrefix = al(kOffState + sizeof(StreamState));
constexpr size_t kOffHist = al(kOffPrefix + 4 * sizeof(int));
constexpr size_t kOffFeat = al(kOffHist + STAB_HBINS * sizeof(unsigned));
constexpr size_t kOffLam = al(kOffFeat + STAB_MAXK * sizeof(float2));
constexpr size_t kOffCand = al(kOffLam + STAB_MAXK * sizeof(float));
constexpr size_t kOffSel = al(kOffCand + kCap * sizeof(unsigned long long));
constexpr size_t kBytes = al(kOffSel + kCap * sizeof(unsigned long long));
constexpr int kChunk = 2048;   // candidates per filter work item (as in the detection kernels)

}  // namespace

// The scratch shared by every call on a device (see the limits above).
static __device__ __align__(256) unsigned char g_detect_scratch[kBytes];

namespace {

// Per-call set-up: the descriptor, the work lists, and the state that must
// start at zero (the histogram and the counters); the candidate arrays are
// overwritten up to their counts and need no clearing.
__global__ void k_noalloc_setup(StreamDev d, int tiles, int chunks)
{
    unsigned char *base = g_detect_scratch;
    unsigned *hist = reinterpret_cast<unsigned *>(base + kOffHist);
    for (int i = threadIdx.x; i < STAB_HBINS; i += blockDim.x) hist[i] = 0u;
    unsigned char *st = base + kOffState;
    for (int i = threadIdx.x; i < (int)sizeof(StreamState); i += blockDim.x) st[i] = 0;
    if (threadIdx.x == 0) {
        *reinterpret_cast<StreamDev *>(base + kOffDesc) = d;
        int *pre = reinterpret_cast<int *>(base + kOffPrefix);
        pre[0] = 0; pre[1] = tiles;    // response tiles
        pre[2] = 0; pre[3] = chunks;   // filter chunks
    }
}

std::mutex g_mu;
unsigned char *g_ptr[256] = {};

// Device address of the scratch array on the current device: looked up once
// per device (host code must not use the symbol itself, which is only a
// host-side stand-in).  The first call on a device also sets the detection
// kernels' launch attributes.
stab_status scratch_address(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return STAB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_detect_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "stab_detect_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return STAB_ERR_CUDA;
        }
        warm_detect();
        g_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_ptr[dev];
    return STAB_OK;
}

}  // namespace

extern "C" stab_status stab_detect_noalloc(const uint8_t *gray, int w, int h, int pitch, int roi_x0, int roi_y0,
                                           int roi_x1, int roi_y1, float quality, int max_corners, float *pts,
                                           float *lam, int *n, int *ncand, void *stream)
{
    if (!gray || !pts || !n || w < 16 || h < 16 || w > 8192 || h > 8192 || pitch < w) return STAB_ERR_INVALID_ARG;
    if (roi_x0 < 3 || roi_y0 < 3 || roi_x1 > w - 3 || roi_y1 > h - 3 || roi_x1 <= roi_x0 || roi_y1 <= roi_y0)
        return STAB_ERR_INVALID_ARG;
    if (max_corners < 1 || !(quality >= 0.f)) return STAB_ERR_INVALID_ARG;
    const int rw = roi_x1 - roi_x0, rh = roi_y1 - roi_y0;
    if (rw > kMaxRoiW || rh > kMaxRoiH || max_corners > STAB_MAXK) {
        fprintf(stderr,
                "stab_detect_noalloc: ROI %d x %d / %d corners exceeds the fixed scratch (ROI <= %d x %d, "
                "corners <= %d)\n",
                rw, rh, max_corners, kMaxRoiW, kMaxRoiH, STAB_MAXK);
        return STAB_ERR_CAPACITY;
    }
    unsigned char *base = nullptr;
    stab_status st = scratch_address(&base);
    if (st != STAB_OK) return st;
    StreamDev d{};
    d.w = w; d.h = h; d.C = 1; d.L = 1; d.K = max_corners;
    d.lw[0] = w; d.lh[0] = h; d.lp[0] = pitch;
    d.period = 1; d.quality = quality;
    d.roi_x0 = roi_x0; d.roi_y0 = roi_y0; d.roi_x1 = roi_x1; d.roi_y1 = roi_y1;
    d.cand_cap = (int)((long long)((rw + 1) / 2) * ((rh + 1) / 2) + 64);
    d.cand = reinterpret_cast<unsigned long long *>(base + kOffCand);
    d.sel = reinterpret_cast<unsigned long long *>(base + kOffSel);
    d.hist = reinterpret_cast<unsigned *>(base + kOffHist);
    d.feat = reinterpret_cast<float2 *>(base + kOffFeat);
    d.det_lam = reinterpret_cast<float *>(base + kOffLam);
    d.st = reinterpret_cast<StreamState *>(base + kOffState);
    const int tiles = stab_resp_items(rw, rh);
    const int chunks = (d.cand_cap + kChunk - 1) / kChunk;
    cudaStream_t s = (cudaStream_t)stream;
    k_noalloc_setup<<<1, 256, 0, s>>>(d, tiles, chunks);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const Launch L{s, sms};
    const StreamDev *S = reinterpret_cast<const StreamDev *>(base + kOffDesc);
    const int *pre = reinterpret_cast<const int *>(base + kOffPrefix);
    DetIO io{gray, pitch, reinterpret_cast<float2 *>(pts), lam, n, ncand};
    launch_begin(L, S, 1, 0, 1);
    launch_response(L, S, WorkList{pre, 1, tiles}, io);
    launch_filter(L, S, WorkList{pre + 2, 1, chunks});
    launch_select(L, S, 1, io);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "stab_detect_noalloc: %s\n", cudaGetErrorString(e));
        return STAB_ERR_CUDA;
    }
    return STAB_OK;
}

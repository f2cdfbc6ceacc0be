// common.cuh -- device-side data layout shared by the kernels of the stabiliser.
//
// One "stream" is one video: its pyramids (two slots, previous and current
// frame), its feature set, its detection scratch, its trajectory ring and (for
// the batched pipeline) its input ring and output frame.  Every kernel walks a
// work list spanning all streams, so one launch serves a whole batch; the
// single-stream API is the same code with n = 1.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "stab.h"

#define STAB_MAXL 8          // pyramid levels
#define STAB_MAXK 2048       // corners per stream
#define STAB_MAXR 12         // LK window radius
// Pyramid slots: frame f lives in slot f mod 3, so a batched step can build
// frame t's pyramid while it tracks frames t-2 -> t-1.
#define STAB_PSLOTS 3
__host__ __device__ inline int stab_pslot(long long f) { return (int)(((f % STAB_PSLOTS) + STAB_PSLOTS) % STAB_PSLOTS); }
#define STAB_CRING 64        // trajectory / motion ring (smoothing window <= 63)
#define STAB_HBINS 4096      // response histogram: top 12 bits of the (non-negative) float score
#define STAB_HSHIFT 19
#define STAB_SEL_SMEM 12288  // selection keys held in shared memory
#define STAB_TW 64           // warp output tile width (pixels)
// Corner response work: strips of 20 rows and 120 columns of the ROI, one warp
// each (lanes 1..30 own 4 columns each; lanes 0 and 31 supply the neighbouring
// columns to lanes 1 and 30), four warps per block.
#define STAB_RS_THREADS 128
// Level-0 work: strips of STAB_L0_ROWS rows and 512 columns (128 threads x 4 columns).
#define STAB_L0_ROWS 24
#define STAB_RS_ROWS 20
#define STAB_RS_COLS 120
__host__ __device__ inline int stab_resp_items(int rw, int rh)
{
    return ((rw + STAB_RS_COLS - 1) / STAB_RS_COLS) * ((rh + STAB_RS_ROWS - 1) / STAB_RS_ROWS);
}
// REDUCE work: a warp owns a strip of stab_pd_rows(h) output rows and
// STAB_PD_COLS output columns (lanes 1..30, 4 columns each; lanes 0 and 31
// compute the neighbouring columns only).  Small levels take shorter strips:
// more warps, each with fewer dependent rows.
#define STAB_PD_COLS 120
__host__ __device__ inline int stab_pd_rows(int h) { return h >= 400 ? 16 : h >= 200 ? 4 : 2; }
__host__ __device__ inline int stab_pd_items(int w, int h)
{
    const int R = stab_pd_rows(h);
    return ((w + STAB_PD_COLS - 1) / STAB_PD_COLS) * ((h + R - 1) / R);
}
#define STAB_WTH 32          // warp output tile: 64 x 32 pixels, 256 threads x 2 rows x 4 pixels

// Per-stream mutable state (device memory).
struct StreamState {
    long long t;          // index of the frame being stepped (0 = first frame)
    int n_feat;           // live features (positions in frame t-1)
    int n_pairs;          // pairs kept by the last track
    int n_cand;           // NMS survivors of the last detection
    int n_sel;            // survivors of the histogram cut
    int blocks_done;      // response CTAs finished (last-CTA threshold step)
    int due;              // detect on frame t-1 during this step
    unsigned lam_max;     // bits of the largest score (scores >= 0 order like unsigned)
    unsigned bin_lo;      // histogram bin where the top-K starts
    unsigned thr_bits;    // bits of quality * max score
    int out_frame[2];     // frame to compose, by the parity of the step whose fit set it (-1 none)
    int err;              // first device error (stab_status), 0 if none
    long long iters;      // LK iterations of this step (statistic)
    long long tpl;        // LK template passes (feature x level x direction) of this step
    unsigned long long fit_key[2];   // best hypothesis so far of the fit in flight, per fitted model
    int fit_ticket;       // fit CTAs of this stream done (the last one refits and clears both)
    int n_det;            // corners of the last detection
    int n_above;          // candidates above the quality threshold (before the top-K cut)
    int hyb_rigid;        // hybrid mechanism: the model held since the last decision (1 rigid)
    int n_due[2];         // stream 0 only: streams due for detection at steps of frame parity 0 / 1
};

struct StreamDev {
    int w, h, C, L, K;
    int lw[STAB_MAXL], lh[STAB_MAXL], lp[STAB_MAXL];   // level sizes, pitch (elements)
    // parameters
    int r, max_iters, period, phase, min_tracks, min_fit, H, model, dwell, W, prec;
    int lag;   // tracking runs this many frames behind the frame being ingested (batches: 1)
    float eps2, min_eig, quality, fb2, tau2, zoom;
    unsigned long long seed;
    int roi_x0, roi_y0, roi_x1, roi_y1;
    // pyramids: two slots (frame parity); u8 levels and I / (Ix, Iy) planes
    uint8_t *u8[STAB_PSLOTS][STAB_MAXL];
    void *pI[STAB_PSLOTS][STAB_MAXL];   // float or __half
    void *pG[STAB_PSLOTS][STAB_MAXL];   // float2 or __half2
    // tracker tensor maps (device memory, 128 bytes each): [slot][level][k],
    // k = 0 template I box, 1 template (Ix, Iy) box, 2 next-frame I box; null
    // when the stream's window radius has no map geometry
    const void *tmap;
    // features and tracks
    float2 *feat;
    float2 *fwd, *back;
    float *fb;
    uint8_t *status, *status_fwd;
    float2 *pair_src, *pair_dst;
    // detection scratch
    unsigned long long *cand;
    int cand_cap;
    unsigned *hist;
    unsigned long long *sel;
    float *det_lam;
    // fit / smoothing
    stab_motion *mring;   // STAB_CRING motions
    float4 *cring;        // STAB_CRING trajectory values
    float *Minv;          // 2 x 8 floats: inverse warps, by the parity of the step whose fit set them
    // batched frames
    uint8_t *ring;
    long long slot_bytes;
    int ring_len, in_pitch;
    uint8_t *out;
    int out_pitch;
    StreamState *st;
};

// A work list: stream i owns items [prefix[i], prefix[i+1]).
struct WorkList {
    const int *prefix;
    int n;
    int total;
    // optional: items handed out by an atomic ticket (ctr[0]) instead of a
    // fixed stride; ctr[1] counts finished groups, and the last resets both
    unsigned *ctr = nullptr;
};

__device__ __forceinline__ int wl_stream(const WorkList &wl, int item)
{
    int lo = 0, hi = wl.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&wl.prefix[mid]) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void set_err(StreamState *st, int code)
{
    atomicCAS(&st->err, 0, code);
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Packed pair of FP32 values (lane 0 in the low word) and the sm_100+ f32x2
// forms of add / sub / fma: each lane is the IEEE operation of its scalar form.
typedef unsigned long long fx2;
__device__ __forceinline__ fx2 pk(float lo, float hi)
{
    fx2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(fx2 v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ fx2 fma2(fx2 a, fx2 b, fx2 c)
{
    fx2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ fx2 add2(fx2 a, fx2 b)
{
    fx2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ fx2 add2_rd(fx2 a, fx2 b)
{
    fx2 d;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ fx2 sub2(fx2 a, fx2 b)
{
    fx2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Plane element access for the two storage precisions.
__device__ __forceinline__ float ld1(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float2 ld2(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ float2 ld2(const __half2 *p) { return __half22float2(__ldg(p)); }

template <typename T> struct Plane2;
template <> struct Plane2<float> { typedef float2 type; };
template <> struct Plane2<__half> { typedef __half2 type; };

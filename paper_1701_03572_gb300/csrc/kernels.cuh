// kernels.cuh -- launch interface between the host runtime and the kernels.
#pragma once

#include <mutex>

#include "common.cuh"

struct Launch {
    cudaStream_t stream;
    int sms;
};

// Once-per-device values (occupancy, kernel attributes).  A function attribute
// set with cudaFuncSetAttribute and an occupancy query apply to the device that
// is current at the time, so each cache keeps one entry per device, filled on
// the first use on that device under a mutex (host threads may drive different
// devices at once).  0 means "not yet computed"; compute() returns >= 1.
constexpr int kMaxDevices = 64;
static inline int current_device()
{
    int d = 0;
    return cudaGetDevice(&d) == cudaSuccess ? d : -1;
}
struct DevCache {
    std::mutex mu;
    int v[kMaxDevices] = {};
    template <class F>
    int get(F &&compute)
    {
        const int d = current_device();
        if (d < 0 || d >= kMaxDevices) return compute();
        std::lock_guard<std::mutex> g(mu);
        if (!v[d]) v[d] = compute();
        return v[d];
    }
};

static inline int grid_for(const Launch &L, int total, int occ)
{
    long long g = (long long)L.sms * (occ < 1 ? 1 : occ);
    if (g > total) g = total;
    if (g < 1) g = 1;
    return (int)g;
}

// Source of level 0: an explicit frame for stream 0 (single-stream calls,
// ptr != NULL) or the stream's input ring slot t % ring (batched step).
struct FrameSrc {
    const uint8_t *ptr;
    int pitch, channels, slot;
};

// Tracker I/O: explicit points and outputs (single-stream test hook) or the
// stream's own feature set and track buffers (pts == NULL).
struct LkIO {
    const float2 *pts;
    int n;
    int slot_prev, slot_next;
    float2 *fwd, *back;
    float *fb;
    uint8_t *status, *status_fwd;
};

// Detection: explicit gray frame (gray != NULL, stream 0) or the previous
// frame's level 0 of each stream when its detection is due.
struct DetIO {
    const uint8_t *gray;
    int pitch;
    float2 *pts_out;
    float *lam_out;
    int *n_out, *ncand_out;
};

struct CompactIO {
    float2 *src_out, *dst_out;
    int *n_out;
    uint8_t *status_out;
};

struct FitIO {
    const float2 *src, *dst;
    const int *n;
    int model;     // stab_model
    long long t;
    stab_motion *out;
};

struct AffineIO {
    const float2 *src, *dst;
    const int *n;
    long long t;
    stab_affine *out;
};

struct WarpIO {
    const uint8_t *src;
    int sp;
    uint8_t *dst;
    int dp, C;
    const float *Minv;
};

void launch_level0(const Launch &L, int prec, const StreamDev *S, WorkList wl, FrameSrc ov);
void launch_pyr_down(const Launch &L, int prec, const StreamDev *S, WorkList wl, int l, int slot_ov);
// Levels l0 .. l1-1 (at most pyr_tail_levels()) in one launch; work items are
// tiles of pyr_tail_tile_w() x pyr_tail_tile_h() pixels of each stream's last
// level below l1 (none for a stream with l0 levels or fewer).
void launch_pyr_tail(const Launch &L, int prec, const StreamDev *S, WorkList wl, int l0, int l1, int slot_ov);
int pyr_tail_tile_w();
int pyr_tail_tile_h();
int pyr_tail_levels();
void warm_pyr_tail();
void launch_plane_f32(const Launch &L, int prec, const StreamDev *S, int slot, int l, float *I, float *Ix,
                      float *Iy);
int occ_level0_f();
int occ_level0_h();
int occ_pyr_f();
int occ_pyr_h();

// Occupancy queries and attributes, done once outside any graph capture.
void warm_detect();
void warm_warp();
void warm_lk();

void launch_begin(const Launch &L, const StreamDev *S, int n, long long t_ov, int force_due);
void launch_response(const Launch &L, const StreamDev *S, WorkList wl, DetIO io);
void launch_filter(const Launch &L, const StreamDev *S, WorkList wl);
void launch_select(const Launch &L, const StreamDev *S, int n, DetIO io);

// Tracker variants (warps per feature, register budget); see k_lk.cu.
int lk_variants();
// Bytes of a stream's tracker tensor maps, and their encoding on the host
// (kLkMapBytes bytes at host_out); returns 0, or -1 if the driver cannot
// encode them.  Only streams with the 21 x 21 window have maps.
constexpr int kLkMapBytes = STAB_PSLOTS * STAB_MAXL * 3 * 128;
int lk_tensor_maps(const StreamDev &D, int prec, void *host_out);
// rcode: the window radius of every stream, or minus the largest when they differ.
void launch_lk(const Launch &L, int prec, int rcode, int variant, const StreamDev *S, WorkList wl, LkIO io);

void launch_compact(const Launch &L, const StreamDev *S, int n, CompactIO io);
void launch_fit(const Launch &L, const StreamDev *S, int n, FitIO io, int streaming, int hmax);
void launch_fit_affine(const Launch &L, const StreamDev *S, AffineIO io);
void launch_smooth_offline(const Launch &L, const stab_motion *m, int T, int W, int w, int h, float zoom,
                           float *mprime, float *Minv);
void launch_smooth_push(const Launch &L, const StreamDev *S, long long t, const stab_motion *m, float *Minv,
                        int *ready);
void launch_advance(const Launch &L, const StreamDev *S, int n);

void launch_warp(const Launch &L, const StreamDev *S, WorkList wl, WarpIO io);

void launch_charb_forward(const Launch &L, const float *It, const float *Ip, int w, int h, int P, float *theta,
                          int margin, float eps, float *loss, float *dtheta, float *gn, int update);
void launch_charb_backward_image(const Launch &L, const float *It, const float *Ip, int w, int h, int P,
                                 const float *theta, int margin, float eps, const float *gout, float *dIt,
                                 float *dIp);

// runtime.cu -- host side of the C ABI declared in include/stab.h.
//
// A Pipeline holds n streams: one device arena carved into every stream's
// buffers, the per-stream descriptors (StreamDev) in device memory, and the
// work lists of each kernel.  The single-stream context is a Pipeline with
// n = 1 driven call by call; the batch enqueues the whole frame step once
// into a CUDA graph and replays it (the per-step frame index lives on the
// device, so the graph never changes).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace {

const char *kVersion = "gb300-stab 0.1 (sm_103a)";

struct Pipeline {
    int n = 0;
    int prec = 0, rmax = 0, rmin = 1 << 30, Lmax = 1, sms = 0, ring = 1;
    std::vector<StreamDev> hs;
    std::vector<stab_params> P;
    StreamDev *ds = nullptr;
    char *arena = nullptr;
    size_t arena_bytes = 0;
    int *prefix = nullptr;
    WorkList wl_l0{}, wl_pyr[STAB_MAXL]{}, wl_tail[STAB_MAXL]{}, wl_resp{}, wl_filter{}, wl_lk{}, wl_warp{};
    std::string err;
    cudaStream_t last = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long t_host = 0;
    int lk_variant = 1;   // tracker kernel variant (autotuned for batches)
    // host-buffer steps: input copies, the step and output copies on three
    // streams chained by events, so copies of neighbouring steps overlap the step
    cudaStream_t hs_in = nullptr, hs_comp = nullptr, hs_out = nullptr;
    // second branch of the step: detection runs beside the pyramid levels >= 1
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_det = nullptr, ev_warp = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_comp[4] = {}, ev_out[4] = {}, ev_join = nullptr;
    bool host_mode = false;   // the last step was a host-buffer step
    std::vector<int> cand_cap0;   // candidate capacity of each stream as sized at creation
    int wmax = 1;             // largest smoothing window of the batch
    int hmax = 1;             // most fit hypotheses of a stream

    // Window radius for the tracker launch: the radius when every stream uses
    // the same one, its negative (the largest) when they differ.
    int rcode() const { return rmin == rmax ? rmax : -rmax; }

    void reset_graph()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
    }

    ~Pipeline()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        for (cudaStream_t x : {hs_in, hs_comp, hs_out, side, side2})
            if (x) cudaStreamDestroy(x);
        for (cudaEvent_t e : {ev_fork, ev_det, ev_warp})
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : {ev_in[0], ev_in[1], ev_comp[0], ev_comp[1], ev_comp[2], ev_comp[3], ev_out[0], ev_out[1],
                              ev_out[2], ev_out[3], ev_join})
            if (e) cudaEventDestroy(e);
        if (prefix) cudaFree(prefix);
        if (ds) cudaFree(ds);
        if (arena) cudaFree(arena);
    }
};

inline int up(int v, int a) { return (v + a - 1) / a * a; }
// A batched step ingests frame t and tracks frames t-2 -> t-1 (the two run as
// parallel branches of the step's graph), so its tracking lags one frame; and
// it composes the frame whose smoothed map the previous step's fit produced.
constexpr int kBatchLag = 1, kWarpLag = 1;

stab_status fail(std::string &err, stab_status code, const std::string &msg)
{
    err = msg;
    return code;
}

stab_status cuda_check(std::string &err, const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return STAB_ERR_CUDA;
    }
    return STAB_OK;
}

stab_status check_params(const stab_params &p, int w, int h, std::string &err)
{
    if (w < 16 || h < 16 || w > 8192 || h > 8192) return fail(err, STAB_ERR_INVALID_ARG, "frame size out of [16, 8192]");
    if (p.max_corners < 1 || p.max_corners > STAB_MAXK) return fail(err, STAB_ERR_INVALID_ARG, "max_corners out of [1, 2048]");
    if (p.levels < 1 || p.levels > STAB_MAXL) return fail(err, STAB_ERR_INVALID_ARG, "levels out of [1, 8]");
    if (p.win_radius < 1 || p.win_radius > STAB_MAXR) return fail(err, STAB_ERR_INVALID_ARG, "win_radius out of [1, 12]");
    if (p.max_iters < 1 || p.max_iters > 1000) return fail(err, STAB_ERR_INVALID_ARG, "max_iters out of [1, 1000]");
    if (!(p.eps >= 0.f) || !(p.min_eig >= 0.f) || !(p.quality >= 0.f) || !(p.fb_thresh >= 0.f) ||
        !(p.inlier_thresh > 0.f))
        return fail(err, STAB_ERR_INVALID_ARG, "negative threshold");
    if (p.redetect_period < 1) return fail(err, STAB_ERR_INVALID_ARG, "redetect_period < 1");
    if (p.redetect_phase < 0 || p.redetect_phase >= p.redetect_period)
        return fail(err, STAB_ERR_INVALID_ARG, "redetect_phase out of [0, redetect_period)");
    if (p.hypotheses < 1 || p.hypotheses > 1 << 20) return fail(err, STAB_ERR_INVALID_ARG, "hypotheses out of range");
    if (p.smooth_window < 1 || p.smooth_window >= STAB_CRING) return fail(err, STAB_ERR_INVALID_ARG, "smooth_window out of [1, 63]");
    if (p.model != STAB_RIGID && p.model != STAB_SIMILARITY && p.model != STAB_HYBRID)
        return fail(err, STAB_ERR_INVALID_ARG, "bad model");
    if (p.dwell < 1) return fail(err, STAB_ERR_INVALID_ARG, "dwell < 1");
    if (!(p.crop_zoom >= 1.f && p.crop_zoom <= 4.f)) return fail(err, STAB_ERR_INVALID_ARG, "crop_zoom out of [1, 4]");
    if (p.precision != STAB_FP32 && p.precision != STAB_FP16_STORAGE) return fail(err, STAB_ERR_INVALID_ARG, "bad precision");
    int lw = w, lh = h;
    for (int l = 1; l < p.levels; ++l) { lw = (lw + 1) / 2; lh = (lh + 1) / 2; }
    if (lw < 2 || lh < 2) return fail(err, STAB_ERR_INVALID_ARG, "too many levels for the frame size");
    int mx = p.roi_margin_x < 0 ? std::max(w / 10, p.win_radius + 2) : p.roi_margin_x;
    int my = p.roi_margin_y < 0 ? std::max(h / 10, p.win_radius + 2) : p.roi_margin_y;
    if (mx < 3 || my < 3 || w - 2 * mx < 1 || h - 2 * my < 1) return fail(err, STAB_ERR_INVALID_ARG, "bad ROI margins");
    return STAB_OK;
}

// Build a pipeline; C[i] = channels of stream i's ring frames (0 = no ring).
stab_status build(Pipeline &pp, int n, const int *w, const int *h, const int *C, const stab_params *P, int ring, int lag)
{
    pp.n = n;
    pp.ring = std::max(ring, 1);
    pp.P.assign(P, P + n);
    pp.hs.assign(n, StreamDev{});
    pp.prec = P[0].precision;
    for (int i = 0; i < n; ++i) {
        stab_status s = check_params(P[i], w[i], h[i], pp.err);
        if (s) return s;
        if (P[i].precision != pp.prec) return fail(pp.err, STAB_ERR_INVALID_ARG, "all streams of a batch share one precision");
        pp.rmax = std::max(pp.rmax, P[i].win_radius);
        pp.rmin = std::min(pp.rmin, P[i].win_radius);
        pp.Lmax = std::max(pp.Lmax, P[i].levels);
        pp.hmax = std::max(pp.hmax, P[i].hypotheses);
    }
    cudaDeviceGetAttribute(&pp.sms, cudaDevAttrMultiProcessorCount, 0);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&pp.sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t psz = pp.prec ? 2 : 4;
    // two passes: size, then carve
    for (int pass = 0; pass < 2; ++pass) {
        size_t off = 0;
        auto take = [&](size_t bytes) -> char * {
            off = (off + 255) & ~size_t(255);
            char *p = pass ? pp.arena + off : nullptr;
            off += bytes;
            return p;
        };
        for (int i = 0; i < n; ++i) {
            StreamDev &D = pp.hs[i];
            const stab_params &p = P[i];
            D.w = w[i]; D.h = h[i]; D.C = C[i] ? C[i] : 1; D.L = p.levels; D.K = p.max_corners;
            D.lw[0] = w[i]; D.lh[0] = h[i];
            for (int l = 1; l < D.L; ++l) { D.lw[l] = (D.lw[l - 1] + 1) / 2; D.lh[l] = (D.lh[l - 1] + 1) / 2; }
            for (int l = 0; l < D.L; ++l) D.lp[l] = up(D.lw[l], 64);
            D.r = p.win_radius; D.max_iters = p.max_iters; D.period = p.redetect_period; D.phase = p.redetect_phase;
            D.min_tracks = p.min_tracks; D.min_fit = p.min_fit; D.H = p.hypotheses;
            D.model = p.model; D.dwell = p.dwell; D.zoom = p.crop_zoom;
            D.W = p.smooth_window; D.prec = p.precision;
            D.eps2 = p.eps * p.eps; D.min_eig = p.min_eig; D.quality = p.quality;
            D.fb2 = p.fb_thresh * p.fb_thresh;
            {
                float tau = p.inlier_thresh;
                volatile float t2 = tau * tau;   // the FP32 product, as the oracle forms it
                D.tau2 = t2;
            }
            D.seed = p.seed;
            int mx = p.roi_margin_x < 0 ? std::max(w[i] / 10, p.win_radius + 2) : p.roi_margin_x;
            int my = p.roi_margin_y < 0 ? std::max(h[i] / 10, p.win_radius + 2) : p.roi_margin_y;
            D.roi_x0 = mx; D.roi_y0 = my; D.roi_x1 = w[i] - mx; D.roi_y1 = h[i] - my;
            D.lag = lag;
            D.tmap = p.win_radius == 10 ? take(kLkMapBytes) : nullptr;
            for (int s = 0; s < STAB_PSLOTS; ++s)
                for (int l = 0; l < D.L; ++l) {
                    size_t px = (size_t)D.lp[l] * D.lh[l];
                    D.u8[s][l] = (uint8_t *)take(px);
                    D.pI[s][l] = take(px * psz);
                    D.pG[s][l] = take(px * psz * 2);
                }
            const size_t K = (size_t)D.K;
            D.feat = (float2 *)take(K * 8);
            D.fwd = (float2 *)take(K * 8);
            D.back = (float2 *)take(K * 8);
            D.fb = (float *)take(K * 4);
            D.status = (uint8_t *)take(K);
            D.status_fwd = (uint8_t *)take(K);
            D.pair_src = (float2 *)take(K * 8);
            D.pair_dst = (float2 *)take(K * 8);
            D.cand_cap = ((D.roi_x1 - D.roi_x0 + 1) / 2) * ((D.roi_y1 - D.roi_y0 + 1) / 2) + 64;
            D.cand = (unsigned long long *)take((size_t)D.cand_cap * 8);
            D.sel = (unsigned long long *)take((size_t)D.cand_cap * 8);
            D.hist = (unsigned *)take(STAB_HBINS * 4);
            D.det_lam = (float *)take(K * 4);
            D.mring = (stab_motion *)take(STAB_CRING * sizeof(stab_motion));
            D.cring = (float4 *)take(STAB_CRING * sizeof(float4));
            D.Minv = (float *)take(16 * 4);
            D.ring_len = pp.ring;
            D.in_pitch = up(D.w * D.C, 64);
            D.slot_bytes = (long long)D.in_pitch * D.h;
            D.out_pitch = D.in_pitch;
            if (C[i]) {
                D.ring = (uint8_t *)take((size_t)D.slot_bytes * pp.ring);
                D.out = (uint8_t *)take((size_t)D.slot_bytes * 2);   // two buffers by step parity
            } else {
                D.ring = nullptr;
                D.out = nullptr;
            }
            D.st = (StreamState *)take(sizeof(StreamState));
        }
        if (!pass) {
            pp.arena_bytes = off;
            if (cudaMalloc(&pp.arena, off) != cudaSuccess) {
                cudaGetLastError();
                pp.arena = nullptr;
                return fail(pp.err, STAB_ERR_OOM, "cudaMalloc of " + std::to_string(off) + " bytes failed");
            }
            if (cudaMemset(pp.arena, 0, off) != cudaSuccess) return cuda_check(pp.err, "cudaMemset");
        }
    }
    // the tracker's tensor maps address the planes just carved
    for (int i = 0; i < n; ++i) {
        StreamDev &D = pp.hs[i];
        if (!D.tmap) continue;
        std::vector<unsigned char> maps(kLkMapBytes);
        if (lk_tensor_maps(D, pp.prec, maps.data()) != 0)
            return fail(pp.err, STAB_ERR_CUDA, "the driver could not encode the tracker's tensor maps");
        if (cudaMemcpy(const_cast<void *>(D.tmap), maps.data(), kLkMapBytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return cuda_check(pp.err, "cudaMemcpy");
    }
    for (int i = 0; i < n; ++i) pp.cand_cap0.push_back(pp.hs[i].cand_cap);
    if (cudaMalloc(&pp.ds, sizeof(StreamDev) * n) != cudaSuccess) return fail(pp.err, STAB_ERR_OOM, "cudaMalloc");
    if (cudaMemcpy(pp.ds, pp.hs.data(), sizeof(StreamDev) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_check(pp.err, "cudaMemcpy");
    // work lists
    std::vector<int> all;
    std::vector<std::pair<WorkList *, std::vector<int>>> lists;
    auto mk = [&](WorkList *wl, auto count) {
        std::vector<int> pre(n + 1, 0);
        for (int i = 0; i < n; ++i) pre[i + 1] = pre[i] + count(pp.hs[i]);
        wl->n = n;
        wl->total = pre[n];
        lists.push_back({wl, pre});
    };
    // level 0: strips of 512 columns x 16 rows (one thread per 4 columns)
    mk(&pp.wl_l0, [](const StreamDev &D) { return ((D.w + 511) / 512) * ((D.h + STAB_L0_ROWS - 1) / STAB_L0_ROWS); });
    for (int l = 1; l < STAB_MAXL; ++l)
        mk(&pp.wl_pyr[l], [l](const StreamDev &D) { return l < D.L ? stab_pd_items(D.lw[l], D.lh[l]) : 0; });
    // levels 2 .. L-1 in groups of pyr_tail_levels(); items are tiles of each
    // stream's last level of the group
    for (int l0 = 2; l0 < STAB_MAXL; l0 += pyr_tail_levels())
        mk(&pp.wl_tail[l0], [l0](const StreamDev &D) {
            if (D.L <= l0) return 0;
            const int lt = std::min(l0 + pyr_tail_levels(), D.L) - 1;
            return ((D.lw[lt] + pyr_tail_tile_w() - 1) / pyr_tail_tile_w()) *
                   ((D.lh[lt] + pyr_tail_tile_h() - 1) / pyr_tail_tile_h());
        });
    mk(&pp.wl_resp, [](const StreamDev &D) { return stab_resp_items(D.roi_x1 - D.roi_x0, D.roi_y1 - D.roi_y0); });
    mk(&pp.wl_filter, [](const StreamDev &D) { return (D.cand_cap + 2047) / 2048; });
    mk(&pp.wl_lk, [](const StreamDev &D) { return D.K; });
    mk(&pp.wl_warp, [](const StreamDev &D) { return ((D.w + STAB_TW - 1) / STAB_TW) * ((D.h + STAB_WTH - 1) / STAB_WTH); });
    for (auto &e : lists) all.insert(all.end(), e.second.begin(), e.second.end());
    all.push_back(0); all.push_back(0);   // the tracker's ticket and finished-group counters
    all.push_back(0); all.push_back(0);   // the corner response's ticket and finished-warp counters
    if (cudaMalloc(&pp.prefix, all.size() * sizeof(int)) != cudaSuccess) return fail(pp.err, STAB_ERR_OOM, "cudaMalloc");
    cudaMemcpy(pp.prefix, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice);
    size_t o = 0;
    for (auto &e : lists) {
        e.first->prefix = pp.prefix + o;
        o += e.second.size();
    }
    // features of unequal cost (iterations, lost tracks) go to whichever group is free
    pp.wl_lk.ctr = reinterpret_cast<unsigned *>(pp.prefix + o);
    pp.wl_resp.ctr = reinterpret_cast<unsigned *>(pp.prefix + o + 2);
    // kernel attributes and occupancy queries happen here, outside any capture
    occ_level0_f(); occ_level0_h(); occ_pyr_f(); occ_pyr_h(); warm_pyr_tail();
    warm_detect(); warm_warp(); warm_lk();
    return cuda_check(pp.err, "create");
}

// Levels >= 1 of pyramid slot `slot` (-1: each stream's slot of its frame
// index): level 1 by the strip kernel, the rest by the fused tile kernel in
// groups of pyr_tail_levels() levels.  prof (optional) marks each launch.
template <typename Mark>
void reduce_levels(Pipeline &pp, const Launch &L, int slot, Mark mark)
{
    static const char *tail_names[STAB_MAXL] = {"", "", "pyr_tail_2", "pyr_tail_3", "pyr_tail_4",
                                                 "pyr_tail_5", "pyr_tail_6", "pyr_tail_7"};
    if (pp.Lmax > 1) {
        launch_pyr_down(L, pp.prec, pp.ds, pp.wl_pyr[1], 1, slot);
        mark("pyr_down_1");
    }
    for (int l0 = 2; l0 < pp.Lmax; l0 += pyr_tail_levels()) {
        launch_pyr_tail(L, pp.prec, pp.ds, pp.wl_tail[l0], l0, std::min(l0 + pyr_tail_levels(), pp.Lmax), slot);
        mark(tail_names[l0]);
    }
}

void build_pyr(Pipeline &pp, const Launch &L, const uint8_t *frame, int pitch, int C, int slot)
{
    launch_level0(L, pp.prec, pp.ds, pp.wl_l0, FrameSrc{frame, pitch, C, slot});
    reduce_levels(pp, L, slot, [](const char *) {});
}

void detect_chain(Pipeline &pp, const Launch &L, DetIO io)
{
    launch_response(L, pp.ds, pp.wl_resp, io);
    launch_filter(L, pp.ds, pp.wl_filter);
    launch_select(L, pp.ds, pp.n, io);
}

// Optional per-kernel event brackets (profiled steps only; never captured).
struct Prof {
    std::vector<std::string> names;
    std::vector<cudaEvent_t> ev;
    cudaStream_t s = nullptr;
    void mark(const char *name)
    {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        ev.push_back(e);
        names.push_back(name ? name : "");
    }
};

void enqueue_step(Pipeline &pp, cudaStream_t s, Prof *pf = nullptr)
{
    Launch L{s, pp.sms};
    auto mark = [&](const char *n) { if (pf) pf->mark(n); };
    mark(nullptr);
    launch_begin(L, pp.ds, pp.n, -1, 0);
    mark("begin");
    if (pf) {   // measured one kernel at a time
        launch_level0(L, pp.prec, pp.ds, pp.wl_l0, FrameSrc{nullptr, 0, 0, 0});
        mark("level0");
        reduce_levels(pp, L, -1, mark);
        launch_response(L, pp.ds, pp.wl_resp, DetIO{});
        mark("response");
        launch_filter(L, pp.ds, pp.wl_filter);
        mark("filter");
        launch_select(L, pp.ds, pp.n, DetIO{});
        mark("select");
        launch_lk(L, pp.prec, pp.rcode(), pp.lk_variant, pp.ds, pp.wl_lk, LkIO{});
        mark("lk");
        launch_compact(L, pp.ds, pp.n, CompactIO{});
        mark("compact");
        launch_fit(L, pp.ds, pp.n, FitIO{}, 1, pp.hmax);
        mark("fit");
        launch_warp(L, pp.ds, pp.wl_warp, WarpIO{});
        mark("warp");
    } else {
        // Three branches that share no buffer: the tracking of frames t-2 -> t-1
        // (detection on frame t-2 when due, tracker, fit, smoothing), the
        // pyramid of frame t (ring slot t, pyramid slot t mod 3), and the
        // composition of the frame whose map the previous step's fit produced.
        const Launch Ls{pp.side, pp.sms}, Lw{pp.side2, pp.sms};
        cudaEventRecord(pp.ev_fork, s);
        cudaStreamWaitEvent(pp.side, pp.ev_fork, 0);
        cudaStreamWaitEvent(pp.side2, pp.ev_fork, 0);
        launch_warp(Lw, pp.ds, pp.wl_warp, WarpIO{});
        cudaEventRecord(pp.ev_warp, pp.side2);
        launch_response(Ls, pp.ds, pp.wl_resp, DetIO{});
        launch_filter(Ls, pp.ds, pp.wl_filter);
        launch_select(Ls, pp.ds, pp.n, DetIO{});
        launch_lk(Ls, pp.prec, pp.rcode(), pp.lk_variant, pp.ds, pp.wl_lk, LkIO{});
        launch_compact(Ls, pp.ds, pp.n, CompactIO{});
        launch_fit(Ls, pp.ds, pp.n, FitIO{}, 1, pp.hmax);
        cudaEventRecord(pp.ev_det, pp.side);
        launch_level0(L, pp.prec, pp.ds, pp.wl_l0, FrameSrc{nullptr, 0, 0, 0});
        reduce_levels(pp, L, -1, [](const char *) {});
        cudaStreamWaitEvent(s, pp.ev_det, 0);
        cudaStreamWaitEvent(s, pp.ev_warp, 0);
    }
    launch_advance(L, pp.ds, pp.n);
    mark("advance");
}

// Bound every stream's candidate list to cap keys (0: the capacity sized at
// creation).  Waits for the pipeline's last stream, then rewrites the field of
// each device descriptor; kernels read it at run time, so a captured graph
// stays valid.
stab_status set_cand_cap(Pipeline &pp, int cap)
{
    if (cap < 0) return fail(pp.err, STAB_ERR_INVALID_ARG, "negative candidate capacity");
    if (cudaStreamSynchronize(pp.last) != cudaSuccess) return cuda_check(pp.err, "stream synchronize");
    for (int i = 0; i < pp.n; ++i) {
        const int c = cap == 0 ? pp.cand_cap0[i] : std::min(cap, pp.cand_cap0[i]);
        pp.hs[i].cand_cap = c;
        if (cudaMemcpy(&pp.ds[i].cand_cap, &c, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            return cuda_check(pp.err, "candidate capacity");
    }
    return STAB_OK;
}

stab_status read_err(Pipeline &pp)
{
    stab_status res = STAB_OK;
    for (int i = 0; i < pp.n; ++i) {
        int e = 0;
        if (cudaMemcpy(&e, &pp.hs[i].st->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return cuda_check(pp.err, "reading the device error word");
        if (e) {
            cudaMemset(&pp.hs[i].st->err, 0, sizeof(int));
            if (res == STAB_OK) {
                res = (stab_status)e;
                pp.err = "device error " + std::to_string(e) + " on stream " + std::to_string(i);
            }
        }
    }
    return res;
}

}  // namespace

struct stab_ctx {
    Pipeline pp;
    long long t_track = 0, t_push = 0;
};

struct stab_batch {
    Pipeline pp;
    std::vector<int> C;
    std::vector<std::string> knames;
};

extern "C" {

const char *stab_version(void) { return kVersion; }

stab_status stab_default_params(stab_params *o)
{
    if (!o) return STAB_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->max_corners = 200;
    o->levels = 3;
    o->win_radius = 10;
    o->max_iters = 30;
    o->eps = 0.01f;
    o->min_eig = 0.01f;
    o->quality = 0.01f;
    o->roi_margin_x = -1;
    o->roi_margin_y = -1;
    o->redetect_period = 5;
    o->min_tracks = 10;
    o->fb_thresh = 1.0f;
    o->inlier_thresh = 1.0f;
    o->hypotheses = 100;
    o->seed = 0;
    o->min_fit = 10;
    o->smooth_window = 15;
    o->model = STAB_SIMILARITY;
    o->precision = STAB_FP32;
    o->dwell = 20;
    o->crop_zoom = 1.0f;
    return STAB_OK;
}

stab_status stab_create(int w, int h, const stab_params *p, stab_ctx **out)
{
    if (!out) return STAB_ERR_INVALID_ARG;
    *out = nullptr;
    stab_params d;
    if (!p) { stab_default_params(&d); p = &d; }
    stab_ctx *c = new stab_ctx();
    int C0 = 0;
    stab_status s = build(c->pp, 1, &w, &h, &C0, p, 1, 0);
    if (s != STAB_OK) {
        fprintf(stderr, "stab_create: %s\n", c->pp.err.c_str());
        delete c;
        return s;
    }
    *out = c;
    return STAB_OK;
}

void stab_destroy(stab_ctx *c)
{
    if (!c) return;
    if (c->pp.last) cudaStreamSynchronize(c->pp.last);
    delete c;
}

const char *stab_last_error(const stab_ctx *c) { return c ? c->pp.err.c_str() : "null context"; }

stab_status stab_sync(stab_ctx *c)
{
    if (!c) return STAB_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(c->pp.last) != cudaSuccess) return cuda_check(c->pp.err, "stream synchronize");
    return read_err(c->pp);
}

#define CTX_LAUNCH(c, stream)                                   \
    Pipeline &pp = (c)->pp;                                     \
    pp.last = (cudaStream_t)(stream);                           \
    Launch L{(cudaStream_t)(stream), pp.sms};

stab_status stab_pyramid(stab_ctx *c, const uint8_t *frame, int pitch, int channels, uint8_t *out, void *stream)
{
    if (!c || !frame || !out || (channels != 1 && channels != 3)) return STAB_ERR_INVALID_ARG;
    if (pitch < c->pp.hs[0].w * channels) return fail(c->pp.err, STAB_ERR_INVALID_ARG, "pitch < w * channels");
    CTX_LAUNCH(c, stream);
    const StreamDev &D = pp.hs[0];
    build_pyr(pp, L, frame, pitch, channels, 0);
    size_t off = 0;
    for (int l = 0; l < D.L; ++l) {
        cudaMemcpy2DAsync(out + off, D.lw[l], D.u8[0][l], D.lp[l], D.lw[l], D.lh[l], cudaMemcpyDeviceToDevice, L.stream);
        off += (size_t)D.lw[l] * D.lh[l];
    }
    return cuda_check(pp.err, "stab_pyramid");
}

stab_status stab_planes(stab_ctx *c, int level, float *I, float *Ix, float *Iy, void *stream)
{
    if (!c || level < 0 || level >= c->pp.hs[0].L) return STAB_ERR_INVALID_ARG;
    CTX_LAUNCH(c, stream);
    launch_plane_f32(L, pp.prec, pp.ds, 0, level, I, Ix, Iy);
    return cuda_check(pp.err, "stab_planes");
}

stab_status stab_detect(stab_ctx *c, const uint8_t *gray, int pitch, float *pts, float *lam, int *n, int *ncand,
                        void *stream)
{
    if (!c || !gray || pitch < c->pp.hs[0].w) return STAB_ERR_INVALID_ARG;
    CTX_LAUNCH(c, stream);
    launch_begin(L, pp.ds, 1, 0, 1);
    detect_chain(pp, L, DetIO{gray, pitch, (float2 *)pts, lam, n, ncand});
    return cuda_check(pp.err, "stab_detect");
}

stab_status stab_lk(stab_ctx *c, const uint8_t *prev, const uint8_t *next, int pitch, const float *pts, int n,
                    float *fwd, float *back, float *fb, uint8_t *status, uint8_t *status_fwd, void *stream)
{
    if (!c || !prev || !next || (n > 0 && (!pts || !fwd || !back || !fb || !status))) return STAB_ERR_INVALID_ARG;
    if (n < 0 || n > c->pp.hs[0].K || pitch < c->pp.hs[0].w) return STAB_ERR_INVALID_ARG;
    CTX_LAUNCH(c, stream);
    build_pyr(pp, L, prev, pitch, 1, 0);
    build_pyr(pp, L, next, pitch, 1, 1);
    if (n > 0) {
        WorkList wl = pp.wl_lk;
        wl.total = n;
        LkIO io{(const float2 *)pts, n, 0, 1, (float2 *)fwd, (float2 *)back, fb, status, status_fwd};
        uint8_t *scratch_status_fwd = nullptr;
        if (!status_fwd) {
            scratch_status_fwd = pp.hs[0].status_fwd;
            io.status_fwd = scratch_status_fwd;
        }
        launch_lk(L, pp.prec, pp.rcode(), pp.lk_variant, pp.ds, wl, io);
    }
    return cuda_check(pp.err, "stab_lk");
}

stab_status stab_track(stab_ctx *c, const uint8_t *prev, const uint8_t *next, int pitch, int channels, int flags,
                       float *pts_prev, float *pts_next, uint8_t *status, int *n, void *stream)
{
    if (!c || !prev || !next || (channels != 1 && channels != 3)) return STAB_ERR_INVALID_ARG;
    if (pitch < c->pp.hs[0].w * channels) return STAB_ERR_INVALID_ARG;
    CTX_LAUNCH(c, stream);
    const long long t = ++c->t_track;
    const int sp = stab_pslot(t - 1), sn = stab_pslot(t);
    if (!(flags & STAB_TRACK_CONTINUE) || t == 1) build_pyr(pp, L, prev, pitch, channels, sp);
    build_pyr(pp, L, next, pitch, channels, sn);
    launch_begin(L, pp.ds, 1, t, 0);
    detect_chain(pp, L, DetIO{});
    launch_lk(L, pp.prec, pp.rcode(), pp.lk_variant, pp.ds, pp.wl_lk, LkIO{});
    launch_compact(L, pp.ds, 1, CompactIO{(float2 *)pts_prev, (float2 *)pts_next, n, status});
    return cuda_check(pp.err, "stab_track");
}

stab_status stab_fit(stab_ctx *c, const float *src, const float *dst, const int *n, int model, int t,
                     stab_motion *out, void *stream)
{
    if (!c || !src || !dst || !n || !out || (model != STAB_RIGID && model != STAB_SIMILARITY && model != STAB_HYBRID))
        return STAB_ERR_INVALID_ARG;
    CTX_LAUNCH(c, stream);
    launch_fit(L, pp.ds, 1, FitIO{(const float2 *)src, (const float2 *)dst, n, model, t, out}, 0, pp.hmax);
    return cuda_check(pp.err, "stab_fit");
}

stab_status stab_fit_affine(stab_ctx *c, const float *src, const float *dst, const int *n, int t, stab_affine *out,
                            void *stream)
{
    if (!c || !src || !dst || !n || !out) return STAB_ERR_INVALID_ARG;
    CTX_LAUNCH(c, stream);
    launch_fit_affine(L, pp.ds, AffineIO{(const float2 *)src, (const float2 *)dst, n, t, out});
    return cuda_check(pp.err, "stab_fit_affine");
}

stab_status stab_smooth(stab_ctx *c, const stab_motion *m, int T, int W, float *mprime, float *Minv, void *stream)
{
    if (!c || !m || !mprime || !Minv || T < 1 || W < 1) return STAB_ERR_INVALID_ARG;
    CTX_LAUNCH(c, stream);
    launch_smooth_offline(L, m, T, W, pp.hs[0].w, pp.hs[0].h, pp.hs[0].zoom, mprime, Minv);
    return cuda_check(pp.err, "stab_smooth");
}

stab_status stab_smooth_push(stab_ctx *c, const stab_motion *m, float *Minv, int *ready, void *stream)
{
    if (!c || !m || !Minv || !ready) return STAB_ERR_INVALID_ARG;
    CTX_LAUNCH(c, stream);
    launch_smooth_push(L, pp.ds, ++c->t_push, m, Minv, ready);
    return cuda_check(pp.err, "stab_smooth_push");
}

stab_status stab_warp(stab_ctx *c, const uint8_t *src, int sp, uint8_t *dst, int dp, int channels, const float *Minv,
                      void *stream)
{
    if (!c || !src || !dst || !Minv || (channels != 1 && channels != 3)) return STAB_ERR_INVALID_ARG;
    if (sp < c->pp.hs[0].w * channels || dp < c->pp.hs[0].w * channels) return STAB_ERR_INVALID_ARG;
    CTX_LAUNCH(c, stream);
    launch_warp(L, pp.ds, pp.wl_warp, WarpIO{src, sp, dst, dp, channels, Minv});
    return cuda_check(pp.err, "stab_warp");
}

// ------------------------------------------------------------------ batch --
stab_status stab_batch_create(int n, const stab_stream_desc *d, int ring, stab_batch **out)
{
    if (!out || n < 1 || n > 4096 || !d) return STAB_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<int> w(n), h(n), C(n);
    std::vector<stab_params> P(n);
    int need = 2;
    for (int i = 0; i < n; ++i) {
        if (d[i].channels != 1 && d[i].channels != 3) return STAB_ERR_INVALID_ARG;
        w[i] = d[i].w; h[i] = d[i].h; C[i] = d[i].channels; P[i] = d[i].params;
        need = std::max(need, P[i].smooth_window / 2 + 2 + kBatchLag + kWarpLag);
    }
    if (ring <= 0) ring = need;
    if (ring < need) return STAB_ERR_INVALID_ARG;
    stab_batch *b = new stab_batch();
    b->C = C;
    stab_status s = build(b->pp, n, w.data(), h.data(), C.data(), P.data(), ring, kBatchLag);
    for (int i = 0; i < n; ++i) b->pp.wmax = std::max(b->pp.wmax, P[i].smooth_window);
    if (s == STAB_OK && (cudaStreamCreateWithFlags(&b->pp.cap, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaStreamCreateWithFlags(&b->pp.side, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaStreamCreateWithFlags(&b->pp.side2, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->pp.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->pp.ev_det, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->pp.ev_warp, cudaEventDisableTiming) != cudaSuccess))
        s = cuda_check(b->pp.err, "stream create");
    if (s != STAB_OK) {
        fprintf(stderr, "stab_batch_create: %s\n", b->pp.err.c_str());
        delete b;
        return s;
    }
    *out = b;
    return STAB_OK;
}

void stab_batch_destroy(stab_batch *b)
{
    if (!b) return;
    if (b->pp.last) cudaStreamSynchronize(b->pp.last);
    delete b;
}

uint8_t *stab_batch_input(stab_batch *b, int i, int slot)
{
    if (!b || i < 0 || i >= b->pp.n || slot < 0 || slot >= b->pp.ring) return nullptr;
    return b->pp.hs[i].ring + (size_t)slot * b->pp.hs[i].slot_bytes;
}

uint8_t *stab_batch_output(stab_batch *b, int i)
{
    if (!b || i < 0 || i >= b->pp.n || !b->pp.hs[i].out) return nullptr;
    const StreamDev &D = b->pp.hs[i];
    return D.out + (size_t)((b->pp.t_host - 1) & 1) * D.slot_bytes;   // the buffer the last step wrote
}

int stab_batch_pitch(const stab_batch *b, int i) { return (b && i >= 0 && i < b->pp.n) ? b->pp.hs[i].in_pitch : 0; }
int stab_batch_ring(const stab_batch *b) { return b ? b->pp.ring : 0; }
int64_t stab_batch_frame(const stab_batch *b) { return b ? b->pp.t_host : -1; }
const char *stab_batch_last_error(const stab_batch *b) { return b ? b->pp.err.c_str() : "null batch"; }

stab_status stab_batch_step(stab_batch *b, int use_graph, void *stream)
{
    if (!b) return STAB_ERR_INVALID_ARG;
    Pipeline &pp = b->pp;
    cudaStream_t s = (cudaStream_t)stream;
    pp.last = s;
    pp.host_mode = false;
    if (use_graph) {
        if (!pp.gexec) {
            if (cudaStreamBeginCapture(pp.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return cuda_check(pp.err, "begin capture");
            enqueue_step(pp, pp.cap);
            if (cudaStreamEndCapture(pp.cap, &pp.graph) != cudaSuccess) return cuda_check(pp.err, "end capture");
            if (cudaGraphInstantiate(&pp.gexec, pp.graph, 0) != cudaSuccess) return cuda_check(pp.err, "instantiate");
        }
        if (cudaGraphLaunch(pp.gexec, s) != cudaSuccess) return cuda_check(pp.err, "graph launch");
    } else {
        enqueue_step(pp, s);
    }
    ++pp.t_host;
    return cuda_check(pp.err, "stab_batch_step");
}

stab_status stab_batch_step_profiled(stab_batch *b, void *stream, float *ms, int n_ms, int *n_kernels)
{
    if (!b || !n_kernels) return STAB_ERR_INVALID_ARG;
    Pipeline &pp = b->pp;
    Prof pf;
    pf.s = (cudaStream_t)stream;
    pp.last = pf.s;
    pp.host_mode = false;
    enqueue_step(pp, pf.s, &pf);
    ++pp.t_host;
    stab_status st = cuda_check(pp.err, "stab_batch_step_profiled");
    cudaStreamSynchronize(pf.s);
    const int nk = (int)pf.ev.size() - 1;
    *n_kernels = nk;
    b->knames.assign(pf.names.begin() + 1, pf.names.end());
    for (int k = 0; k < nk && ms && k < n_ms; ++k) {
        float v = 0.f;
        cudaEventElapsedTime(&v, pf.ev[k], pf.ev[k + 1]);
        ms[k] = v;
    }
    for (auto e : pf.ev) cudaEventDestroy(e);
    if (st == STAB_OK) st = cuda_check(pp.err, "stab_batch_step_profiled");
    return st;
}

const char *stab_batch_kernel_name(const stab_batch *b, int i)
{
    if (!b || i < 0 || i >= (int)b->knames.size()) return "";
    return b->knames[i].c_str();
}

stab_status stab_batch_lk_work(stab_batch *b, int64_t *iterations, int64_t *templates)
{
    if (!b || !iterations || !templates) return STAB_ERR_INVALID_ARG;
    Pipeline &pp = b->pp;
    if (cudaStreamSynchronize(pp.last) != cudaSuccess) return cuda_check(pp.err, "stream synchronize");
    *iterations = 0;
    *templates = 0;
    for (int i = 0; i < pp.n; ++i) {
        long long it = 0, tp = 0;
        cudaMemcpy(&it, &pp.hs[i].st->iters, sizeof(it), cudaMemcpyDeviceToHost);
        cudaMemcpy(&tp, &pp.hs[i].st->tpl, sizeof(tp), cudaMemcpyDeviceToHost);
        *iterations += it;
        *templates += tp;
    }
    return cuda_check(pp.err, "stab_batch_lk_work");
}

stab_status stab_set_candidate_capacity(stab_ctx *c, int cap)
{
    if (!c) return STAB_ERR_INVALID_ARG;
    return set_cand_cap(c->pp, cap);
}

stab_status stab_batch_set_candidate_capacity(stab_batch *b, int cap)
{
    if (!b) return STAB_ERR_INVALID_ARG;
    return set_cand_cap(b->pp, cap);
}

int stab_lk_variants(void) { return lk_variants(); }

stab_status stab_set_lk_variant(stab_ctx *c, int v)
{
    if (!c || v < 0 || v >= lk_variants()) return STAB_ERR_INVALID_ARG;
    c->pp.lk_variant = v;
    return STAB_OK;
}

stab_status stab_batch_set_lk_variant(stab_batch *b, int v)
{
    if (!b || v < 0 || v >= lk_variants()) return STAB_ERR_INVALID_ARG;
    if (b->pp.lk_variant != v) {
        b->pp.lk_variant = v;
        b->pp.reset_graph();
    }
    return STAB_OK;
}

static std::string batch_signature(const Pipeline &pp)
{
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::string sig = std::string(prop.name) + "|prec" + std::to_string(pp.prec) + "|r" + std::to_string(pp.rmax);
    for (const auto &D : pp.hs)
        sig += "|" + std::to_string(D.w) + "x" + std::to_string(D.h) + "x" + std::to_string(D.C) + "k" +
               std::to_string(D.K) + "l" + std::to_string(D.L);
    for (auto &ch : sig)
        if (ch == '"' || ch == '\\') ch = '_';
    return sig;
}

// Cache file: one JSON object {"signature": variant, ...}, written only here.
static bool cache_lookup(const char *path, const std::string &sig, int *v)
{
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    std::string txt;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, k);
    fclose(f);
    const std::string key = "\"" + sig + "\":";
    size_t pos = txt.find(key);
    if (pos == std::string::npos) return false;
    *v = atoi(txt.c_str() + pos + key.size());
    return *v >= 0 && *v < lk_variants();
}

static void cache_store(const char *path, const std::string &sig, int v)
{
    if (!path) return;
    std::vector<std::pair<std::string, int>> ent;
    if (FILE *f = fopen(path, "r")) {
        std::string txt;
        char buf[4096];
        size_t k;
        while ((k = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, k);
        fclose(f);
        size_t p = 0;
        while ((p = txt.find('"', p)) != std::string::npos) {
            size_t q = txt.find('"', p + 1);
            if (q == std::string::npos) break;
            std::string key = txt.substr(p + 1, q - p - 1);
            size_t c = txt.find(':', q);
            if (c == std::string::npos) break;
            if (key != sig) ent.push_back({key, atoi(txt.c_str() + c + 1)});
            p = txt.find_first_of(",}", c);
            if (p == std::string::npos) break;
        }
    }
    ent.push_back({sig, v});
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    for (size_t i = 0; i < ent.size(); ++i)
        fprintf(f, "  \"%s\": %d%s\n", ent[i].first.c_str(), ent[i].second, i + 1 < ent.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

stab_status stab_batch_autotune(stab_batch *b, const char *cache_path, int *variant, float *ms_out, void *stream)
{
    if (!b) return STAB_ERR_INVALID_ARG;
    Pipeline &pp = b->pp;
    if (pp.t_host < 2 + kBatchLag)
        return fail(pp.err, STAB_ERR_INVALID_ARG, "autotune needs the batch to have run three steps");
    const std::string sig = batch_signature(pp);
    int v = -1;
    const int nv = lk_variants();
    if (ms_out)
        for (int i = 0; i < nv; ++i) ms_out[i] = -1.f;
    if (!cache_lookup(cache_path, sig, &v)) {
        cudaStream_t s = (cudaStream_t)stream;
        Launch L{s, pp.sms};
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (int cand = 0; cand < nv; ++cand) {
            // the tracker reads the features and pyramids of the last step and
            // writes only its own outputs, so repeated launches are harmless
            launch_lk(L, pp.prec, pp.rcode(), cand, pp.ds, pp.wl_lk, LkIO{});
            cudaEventRecord(e0, s);
            for (int k = 0; k < 5; ++k) launch_lk(L, pp.prec, pp.rcode(), cand, pp.ds, pp.wl_lk, LkIO{});
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 5.f;
            if (ms_out) ms_out[cand] = ms;
            if (ms < best) { best = ms; v = cand; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        stab_status st = cuda_check(pp.err, "stab_batch_autotune");
        if (st != STAB_OK) return st;
        cache_store(cache_path, sig, v);
    }
    if (variant) *variant = v;
    return stab_batch_set_lk_variant(b, v);
}

static stab_status host_streams(Pipeline &pp)
{
    if (pp.hs_in) return STAB_OK;
    bool ok = cudaStreamCreateWithFlags(&pp.hs_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&pp.hs_comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&pp.hs_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&pp.ev_join, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < 4; ++k)
        ok = cudaEventCreateWithFlags(&pp.ev_comp[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&pp.ev_out[k], cudaEventDisableTiming) == cudaSuccess &&
             (k >= 2 || cudaEventCreateWithFlags(&pp.ev_in[k], cudaEventDisableTiming) == cudaSuccess);
    return ok ? STAB_OK : cuda_check(pp.err, "host-step streams");
}

// Host-buffer step t: copies of frame t into ring slot t % ring on hs_in, the
// step on hs_comp, copies of the composed frames on hs_out, chained by events.
// Slot t % ring is last read by the warp of step t - ring + 3 + W/2 (the warp
// composes frame t - 3 - W/2), done once step t - 2 is done when
// ring >= W/2 + 5 (else the copies wait for step t - 1);
// the output buffer of step t (parity t) was last read by the output copies
// of step t - 2.  The caller's stream waits for this step's output copies.
stab_status stab_batch_step_host(stab_batch *b, const uint8_t *const *frames, uint8_t *const *outs, void *stream)
{
    if (!b || !frames) return STAB_ERR_INVALID_ARG;
    for (int i = 0; i < b->pp.n; ++i)
        if (!frames[i]) return STAB_ERR_INVALID_ARG;
    Pipeline &pp = b->pp;
    stab_status st = host_streams(pp);
    if (st != STAB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const long long t = pp.t_host;
    if (!pp.host_mode) {   // order after whatever the caller submitted before
        cudaEventRecord(pp.ev_join, s);
        cudaStreamWaitEvent(pp.hs_in, pp.ev_join, 0);
        cudaStreamWaitEvent(pp.hs_comp, pp.ev_join, 0);
        cudaStreamWaitEvent(pp.hs_out, pp.ev_join, 0);
    }
    const long long back = pp.ring >= pp.wmax / 2 + kBatchLag + kWarpLag + 3 ? 2 : 1;
    if (pp.host_mode && t >= back) cudaStreamWaitEvent(pp.hs_in, pp.ev_comp[(t - back) & 3], 0);
    for (int i = 0; i < pp.n; ++i) {
        const StreamDev &D = pp.hs[i];
        cudaMemcpy2DAsync(D.ring + (size_t)(t % pp.ring) * D.slot_bytes, D.in_pitch, frames[i], (size_t)D.w * D.C,
                          (size_t)D.w * D.C, D.h, cudaMemcpyHostToDevice, pp.hs_in);
    }
    cudaEventRecord(pp.ev_in[t & 1], pp.hs_in);
    cudaStreamWaitEvent(pp.hs_comp, pp.ev_in[t & 1], 0);
    if (pp.host_mode && t >= 2) cudaStreamWaitEvent(pp.hs_comp, pp.ev_out[(t - 2) & 3], 0);
    st = stab_batch_step(b, 1, pp.hs_comp);
    if (st != STAB_OK) return st;
    cudaEventRecord(pp.ev_comp[t & 3], pp.hs_comp);
    cudaStreamWaitEvent(pp.hs_out, pp.ev_comp[t & 3], 0);
    if (outs)
        for (int i = 0; i < pp.n; ++i) {
            const StreamDev &D = pp.hs[i];
            if (outs[i] && t - kBatchLag - kWarpLag - 1 - pp.P[i].smooth_window / 2 >= 0)
                cudaMemcpy2DAsync(outs[i], (size_t)D.w * D.C, D.out + (size_t)(t & 1) * D.slot_bytes, D.out_pitch,
                                  (size_t)D.w * D.C, D.h, cudaMemcpyDeviceToHost, pp.hs_out);
        }
    cudaEventRecord(pp.ev_out[t & 3], pp.hs_out);
    cudaStreamWaitEvent(s, pp.ev_out[t & 3], 0);
    pp.last = s;
    pp.host_mode = true;
    return cuda_check(pp.err, "stab_batch_step_host");
}

stab_status stab_batch_sync(stab_batch *b)
{
    if (!b) return STAB_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->pp.last) != cudaSuccess) return cuda_check(b->pp.err, "stream synchronize");
    return read_err(b->pp);
}

stab_status stab_batch_motions(stab_batch *b, stab_motion *out)
{
    if (!b || !out) return STAB_ERR_INVALID_ARG;
    Pipeline &pp = b->pp;
    if (cudaStreamSynchronize(pp.last) != cudaSuccess) return cuda_check(pp.err, "stream synchronize");
    const long long t = pp.t_host - 1 - kBatchLag;   // transition tracked by the last step
    for (int i = 0; i < pp.n; ++i) {
        if (t < 0) { std::memset(&out[i], 0, sizeof(stab_motion)); continue; }
        cudaMemcpy(&out[i], pp.hs[i].mring + (t % STAB_CRING), sizeof(stab_motion), cudaMemcpyDeviceToHost);
    }
    return cuda_check(pp.err, "stab_batch_motions");
}

stab_status stab_batch_features(stab_batch *b, int i, float *pts, int *n)
{
    if (!b || i < 0 || i >= b->pp.n || !pts || !n) return STAB_ERR_INVALID_ARG;
    Pipeline &pp = b->pp;
    if (cudaStreamSynchronize(pp.last) != cudaSuccess) return cuda_check(pp.err, "stream synchronize");
    cudaMemcpy(n, &pp.hs[i].st->n_feat, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(pts, pp.hs[i].feat, sizeof(float2) * pp.hs[i].K, cudaMemcpyDeviceToHost);
    return cuda_check(pp.err, "stab_batch_features");
}

// ------------------------------------------------- photometric refinement --
static stab_status charb_args(const float *It, const float *Ip, int w, int h, int P, const void *theta, int margin,
                              float eps)
{
    if (!It || !Ip || !theta || w < 4 || h < 4 || P < 1 || P > (1 << 20) || margin < 0 || 2 * margin >= w ||
        2 * margin >= h || !(eps > 0.f))
        return STAB_ERR_INVALID_ARG;
    return STAB_OK;
}

static Launch plain_launch(void *stream)
{
    static DevCache c;
    const int sms = c.get([] {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, current_device());
        return n > 0 ? n : 1;
    });
    return Launch{(cudaStream_t)stream, sms};
}

stab_status stab_charb_forward(const float *It, const float *Ip, int w, int h, int P, const float *theta, int margin,
                               float eps, float *loss, float *dtheta, float *gn, void *stream)
{
    stab_status st = charb_args(It, Ip, w, h, P, theta, margin, eps);
    if (st) return st;
    std::string err;
    launch_charb_forward(plain_launch(stream), It, Ip, w, h, P, const_cast<float *>(theta), margin, eps, loss, dtheta,
                         gn, 0);
    return cuda_check(err, "stab_charb_forward");
}

stab_status stab_charb_backward_image(const float *It, const float *Ip, int w, int h, int P, const float *theta,
                                      int margin, float eps, const float *gout, float *dIt, float *dIp, void *stream)
{
    stab_status st = charb_args(It, Ip, w, h, P, theta, margin, eps);
    if (st) return st;
    if (!dIt && !dIp) return STAB_ERR_INVALID_ARG;
    std::string err;
    launch_charb_backward_image(plain_launch(stream), It, Ip, w, h, P, theta, margin, eps, gout, dIt, dIp);
    return cuda_check(err, "stab_charb_backward_image");
}

stab_status stab_charb_gauss_newton(const float *It, const float *Ip, int w, int h, int P, float *theta, int margin,
                                    float eps, int steps, void *stream)
{
    stab_status st = charb_args(It, Ip, w, h, P, theta, margin, eps);
    if (st) return st;
    if (steps < 0 || steps > 1000) return STAB_ERR_INVALID_ARG;
    std::string err;
    const Launch L = plain_launch(stream);
    for (int k = 0; k < steps; ++k)
        launch_charb_forward(L, It, Ip, w, h, P, theta, margin, eps, nullptr, nullptr, nullptr, 1);
    return cuda_check(err, "stab_charb_gauss_newton");
}

}  // extern "C"

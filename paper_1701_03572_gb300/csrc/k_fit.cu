// k_fit.cu -- pair compaction, robust rigid / similarity fit (Sec. 4 and 4.1,
// Eq. 7 restricted to 3 or 4 degrees of freedom) and the averaging-window
// trajectory smoothing of Sec. 5.1 (offline over a clip, or streaming with a
// W/2-frame lookahead, the GPU form of the paper's motion-compensation thread).
//
// The fit runs up to 8 CTAs per stream, each scoring a slice of the
// hypotheses; the last to finish refits on the overall winner.  Hypothesis h
// draws its two-point sample from the SplitMix64 hash of (seed, t, h) and is
// scored by its inlier count; model and residual use one fixed IEEE FP32
// operation sequence (explicit _rn intrinsics, no contraction), so counts and
// the winning hypothesis are reproducible bit for bit.  The closed-form
// least-squares refit on the winner's inliers uses fixed-order FP32 block
// reductions.  With the hybrid mechanism (Sec. 4.1) a decision transition fits
// both models in the same launch and keeps the rigid one iff its RMS over its
// own inliers is strictly lower; the choice is held in the stream state until
// the next decision.
#include "kernels.cuh"

namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// r mod n for 64-bit r without a 64-bit division per call: with m = floor((2^64
// - 1) / n), q = floor(r m / 2^64) satisfies r/n - 3 < q <= r/n, so r - q n lies
// in [0, 3n) and at most two subtractions finish it (the result is exact).
struct Mod64 { unsigned long long m, n; };
__device__ __forceinline__ Mod64 mod64_of(unsigned long long n) { return Mod64{~0ull / n, n}; }
__device__ __forceinline__ unsigned long long mod64(unsigned long long r, const Mod64 &d)
{
    unsigned long long x = r - __umul64hi(r, d.m) * d.n;
    while (x >= d.n) x -= d.n;
    return x;
}

// mn: modulus n, mn1: modulus n - 1 (n >= 2 staged pairs)
__device__ __forceinline__ void sample_pair(unsigned long long seed, long long t, int h, const Mod64 &mn,
                                            const Mod64 &mn1, int &i, int &j)
{
    unsigned long long base = seed ^ ((unsigned long long)(unsigned)t << 32) ^ ((unsigned long long)(unsigned)h << 8);
    unsigned long long r0 = splitmix64(base), r1 = splitmix64(base ^ 1ull);
    i = (int)mod64(r0, mn);
    int b = (int)mod64(r1, mn1);
    j = b >= i ? b + 1 : b;
}

// d = [a -b; b a] s + (m2, m3), through (si, di) and (sj, dj)
__device__ __forceinline__ bool two_point(float2 si, float2 sj, float2 di, float2 dj, int rigid, float m[4])
{
    const float vsx = __fsub_rn(sj.x, si.x), vsy = __fsub_rn(sj.y, si.y);
    const float vdx = __fsub_rn(dj.x, di.x), vdy = __fsub_rn(dj.y, di.y);
    const float nn = __fmaf_rn(vsx, vsx, __fmul_rn(vsy, vsy));
    if (!(nn >= 1.0f)) return false;
    const float dot = __fmaf_rn(vsx, vdx, __fmul_rn(vsy, vdy));
    const float crs = __fmaf_rn(vsx, vdy, -__fmul_rn(vsy, vdx));
    float a, b;
    if (rigid) {
        const float rr = __fsqrt_rn(__fmaf_rn(dot, dot, __fmul_rn(crs, crs)));
        if (!(rr > 0.0f)) return false;
        a = __fdiv_rn(dot, rr); b = __fdiv_rn(crs, rr);
    } else {
        a = __fdiv_rn(dot, nn); b = __fdiv_rn(crs, nn);
    }
    const float msx = __fmul_rn(0.5f, __fadd_rn(si.x, sj.x)), msy = __fmul_rn(0.5f, __fadd_rn(si.y, sj.y));
    const float mdx = __fmul_rn(0.5f, __fadd_rn(di.x, dj.x)), mdy = __fmul_rn(0.5f, __fadd_rn(di.y, dj.y));
    m[0] = a; m[1] = b;
    m[2] = __fsub_rn(mdx, __fmaf_rn(a, msx, -__fmul_rn(b, msy)));
    m[3] = __fsub_rn(mdy, __fmaf_rn(b, msx, __fmul_rn(a, msy)));
    return true;
}

__device__ __forceinline__ bool is_inlier(const float m[4], float2 s, float2 d, float tau2)
{
    const float px = __fmaf_rn(m[0], s.x, __fmaf_rn(-m[1], s.y, m[2]));
    const float py = __fmaf_rn(m[1], s.x, __fmaf_rn(m[0], s.y, m[3]));
    const float ex = __fsub_rn(d.x, px), ey = __fsub_rn(d.y, py);
    return __fmaf_rn(ex, ex, __fmul_rn(ey, ey)) < tau2;
}

// Fixed-order sum of NV values over the block (512 threads = 16 warps).
template <int NV>
__device__ __forceinline__ void block_sum(float v[NV], float (*sred)[NV])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < NV; ++k) sred[wid][k] = v[k];
    __syncthreads();
    for (int k = 0; k < NV; ++k) {
        float a = 0.f;
        for (int i = 0; i < nw; ++i) a += sred[i][k];
        v[k] = a;
    }
    __syncthreads();
}

// Stable compaction of kept tracks: pairs (src = feature, dst = forward
// result) in feature order; the kept destinations become the next features.
__global__ void __launch_bounds__(1024) k_compact(const StreamDev *__restrict__ S, CompactIO io)
{
    __shared__ int wsum_[32];
    const StreamDev &D = S[blockIdx.x];
    StreamState *st = D.st;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int n = st->t - D.lag >= 1 ? st->n_feat : 0;
    // two consecutive features per thread (K <= 2048)
    const int f0 = 2 * tid;
    const int k0 = (f0 < n) && D.status[f0], k1 = (f0 + 1 < n) && D.status[f0 + 1];
    const float2 s0 = k0 ? D.feat[f0] : make_float2(0, 0), s1 = k1 ? D.feat[f0 + 1] : make_float2(0, 0);
    const float2 d0 = k0 ? D.fwd[f0] : make_float2(0, 0), d1 = k1 ? D.fwd[f0 + 1] : make_float2(0, 0);
    int c = k0 + k1, incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum_[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int v = wsum_[lane], x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        wsum_[lane] = x - v;   // exclusive prefix of warp totals
    }
    __syncthreads();
    int pos = wsum_[wid] + incl - c;
    if (k0) { D.pair_src[pos] = s0; D.pair_dst[pos] = d0; ++pos; }
    if (k1) { D.pair_src[pos] = s1; D.pair_dst[pos] = d1; }
    if (io.status_out) {
        if (f0 < D.K) io.status_out[f0] = (uint8_t)k0;
        if (f0 + 1 < D.K) io.status_out[f0 + 1] = (uint8_t)k1;
    }
    __shared__ int s_total;
    if (tid == blockDim.x - 1) s_total = wsum_[wid] + incl;
    __syncthreads();
    const int m = s_total;
    for (int i = tid; i < m; i += blockDim.x) {
        float2 sv = D.pair_src[i], dv = D.pair_dst[i];
        D.feat[i] = dv;
        if (io.src_out) io.src_out[i] = sv;
        if (io.dst_out) io.dst_out[i] = dv;
    }
    if (tid == 0) {
        st->n_pairs = m;
        st->n_feat = m;
        if (io.n_out) *io.n_out = m;
    }
}

// Streaming smoothing step for frame t with motion m (thread-local; one
// thread per stream).  C_t = C_{t-1} + m_t; when frame u = t - 1 - W/2 >= 0 is
// ready: S = mean of C over [max(0, u+1 - (W-1)/2), t], m' = m_{u+1} + (S -
// C_{u+1}), inverse warp of m'.
// Composition crop (Sec. 5.1): a zoom z about the centre applied to the
// output, q = W(c + (p - c) / z) with W the inverse warp of m', which is the
// inverse warp of (z tx, z ty, theta, log s + log z).
__device__ void inverse_warp(float4 mp, int w, int h, float zoom, float *Minv)
{
    const float cx = 0.5f * (float)(w - 1), cy = 0.5f * (float)(h - 1);
    const float is = __fdiv_rn(expf(-mp.w), zoom);
    float sn, c;
    sincosf(mp.z, &sn, &c);
    const float a00 = is * c, a01 = is * sn, a10 = -is * sn, a11 = is * c;
    const float ux = cx + zoom * mp.x, uy = cy + zoom * mp.y;
    Minv[0] = a00; Minv[1] = a01; Minv[2] = cx - (a00 * ux + a01 * uy);
    Minv[3] = a10; Minv[4] = a11; Minv[5] = cy - (a10 * ux + a11 * uy);
}

__device__ __forceinline__ float4 add4(float4 a, float4 b)
{
    return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
}

__device__ __forceinline__ float4 corrected(float4 m, float4 S, float4 C)
{
    return make_float4(__fadd_rn(m.x, __fsub_rn(S.x, C.x)), __fadd_rn(m.y, __fsub_rn(S.y, C.y)),
                       __fadd_rn(m.z, __fsub_rn(S.z, C.z)), __fadd_rn(m.w, __fsub_rn(S.w, C.w)));
}

__device__ __forceinline__ float4 mot4(const stab_motion &m) { return make_float4(m.tx, m.ty, m.theta, m.log_scale); }

// Called by the 32 lanes of one warp.  Lane 0 appends C_t; the lanes then load
// the window's trajectory entries together and every lane sums them in the
// order k = lo .. t (the offline smoother's order, so both emit the same
// bits); lane 0 writes the inverse warp.  Returns u (or -1) on every lane.
__device__ int smooth_step(stab_motion *mring, float4 *cring, long long t, int W, int w, int h, float zoom,
                           float *Minv)
{
    const int CR = STAB_CRING, lane = threadIdx.x & 31;
    if (lane == 0) {
        const float4 Cp = t > 0 ? cring[(t - 1) % CR] : make_float4(0.f, 0.f, 0.f, 0.f);
        cring[t % CR] = add4(Cp, mot4(mring[t % CR]));
    }
    __syncwarp();
    const long long u = t - 1 - W / 2;
    if (u < 0) return -1;
    const long long j = u + 1;
    long long lo = j - (W - 1) / 2;
    if (lo < 0) lo = 0;
    const int n = (int)(t - lo + 1);   // <= W < CR
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 v0 = lane < n ? cring[(lo + lane) % CR] : z;
    const float4 v1 = lane + 32 < n ? cring[(lo + lane + 32) % CR] : z;
    float4 acc = z;
    for (int k = 0; k < n; ++k) {
        const float4 src = k < 32 ? v0 : v1;
        const float4 x = make_float4(__shfl_sync(0xffffffffu, src.x, k & 31), __shfl_sync(0xffffffffu, src.y, k & 31),
                                     __shfl_sync(0xffffffffu, src.z, k & 31), __shfl_sync(0xffffffffu, src.w, k & 31));
        acc = add4(acc, x);
    }
    const float cnt = (float)n;
    const float4 Sm = make_float4(__fdiv_rn(acc.x, cnt), __fdiv_rn(acc.y, cnt), __fdiv_rn(acc.z, cnt),
                                  __fdiv_rn(acc.w, cnt));
    if (lane == 0) inverse_warp(corrected(mot4(mring[j % CR]), Sm, cring[j % CR]), w, h, zoom, Minv);
    return (int)u;
}

struct FitRes {
    float tx, ty, th, ls, rms;
    int inliers;
    bool ok;
};

struct FitShared {
    unsigned long long key[16];   // per-warp best hypotheses (score_slice)
    float red[16][5];
};

// Hypothesis scoring of one model for a slice of the hypotheses: warp g of
// the stream's G scoring warps takes h = g, g + G, ...; a hypothesis scores its
// inlier count (-1 when its two points are degenerate).  The block's best as
// a key, larger = more inliers, then the lower h (the first best):
// (count + 1) << 32 | ~h.  Every thread of the block returns it.
__device__ __forceinline__ unsigned long long fit_key(int cnt, int h)
{
    return ((unsigned long long)(unsigned)(cnt + 1) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)h);
}

__device__ unsigned long long score_slice(const float2 *ss, const float2 *sd, int n, int rigid, const StreamDev &D,
                                          long long t, int g, int G, const Mod64 &mn, const Mod64 &mn1,
                                          unsigned long long *skey)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int best = -1, bh = 0x7fffffff;
    for (int hh = g; hh < D.H; hh += G) {
        int i, j;
        sample_pair(D.seed, t, hh, mn, mn1, i, j);
        float m[4];
        int cnt = -1;
        if (two_point(ss[i], ss[j], sd[i], sd[j], rigid, m)) {
            int c = 0;
            for (int k = lane; k < n; k += 32) c += is_inlier(m, ss[k], sd[k], D.tau2);
            cnt = __reduce_add_sync(0xffffffffu, c);
        }
        if (cnt > best) { best = cnt; bh = hh; }
    }
    __syncthreads();   // earlier readers of skey are done
    if (lane == 0) skey[wid] = fit_key(best, bh);
    __syncthreads();
    unsigned long long k = 0;
    for (int w = 0; w < nwarps; ++w) k = max(k, skey[w]);
    return k;
}

// Least-squares refit of one model on the inliers of the winning hypothesis
// (key from score_slice over all of the stream's hypotheses): the closed-form
// similarity / rigid fit and the RMS residual of those inliers.
__device__ FitRes refit(const float2 *ss, const float2 *sd, int n, int rigid, const StreamDev &D, long long t,
                        unsigned long long key, const Mod64 &mn, const Mod64 &mn1, FitShared &sh)
{
    const int tid = threadIdx.x;
    FitRes r;
    r.ok = false;
    r.tx = r.ty = r.th = r.ls = r.rms = 0.f;
    r.inliers = 0;
    const int best = (int)(unsigned)(key >> 32) - 1, bh = (int)(0xFFFFFFFFu - (unsigned)key);
    if (best < 2) return r;
    int i, j;
    sample_pair(D.seed, t, bh, mn, mn1, i, j);
    float m[4];
    two_point(ss[i], ss[j], sd[i], sd[j], rigid, m);
    float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = tid; k < n; k += blockDim.x)
        if (is_inlier(m, ss[k], sd[k], D.tau2)) {
            v[0] += 1.f; v[1] += ss[k].x; v[2] += ss[k].y; v[3] += sd[k].x; v[4] += sd[k].y;
        }
    block_sum<5>(v, sh.red);
    const float ni = v[0];
    const float msx = v[1] / ni, msy = v[2] / ni, mdx = v[3] / ni, mdy = v[4] / ni;
    float u[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = tid; k < n; k += blockDim.x)
        if (is_inlier(m, ss[k], sd[k], D.tau2)) {
            const float x0 = ss[k].x - msx, x1 = ss[k].y - msy;
            const float y0 = sd[k].x - mdx, y1 = sd[k].y - mdy;
            u[0] += x0 * y0 + x1 * y1;
            u[1] += x0 * y1 - x1 * y0;
            u[2] += x0 * x0 + x1 * x1;
        }
    block_sum<5>(u, sh.red);
    if (!(u[2] > 0.f)) return r;
    const float th = atan2f(u[1], u[0]);
    const float sc = rigid ? 1.f : sqrtf(u[0] * u[0] + u[1] * u[1]) / u[2];
    float sn, c;
    sincosf(th, &sn, &c);
    const float tx = mdx - sc * (c * msx - sn * msy);
    const float ty = mdy - sc * (sn * msx + c * msy);
    float e[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = tid; k < n; k += blockDim.x)
        if (is_inlier(m, ss[k], sd[k], D.tau2)) {
            const float px = sc * (c * ss[k].x - sn * ss[k].y) + tx;
            const float py = sc * (sn * ss[k].x + c * ss[k].y) + ty;
            e[0] += (sd[k].x - px) * (sd[k].x - px) + (sd[k].y - py) * (sd[k].y - py);
        }
    block_sum<5>(e, sh.red);
    r.tx = tx; r.ty = ty; r.th = th; r.ls = logf(sc);
    r.inliers = (int)ni;
    r.rms = sqrtf(e[0] / ni);
    r.ok = true;
    return r;
}

// Grid (streams, parts): the parts of a stream each stage its pairs and score
// a slice of its hypotheses, folding their best into the stream's key with an
// atomic maximum; the last part to finish (ticket) reads and clears the keys,
// refits, decides and smooths.
__global__ void __launch_bounds__(512) k_fit(const StreamDev *__restrict__ S, FitIO io, int streaming)
{
    __shared__ float2 ss[STAB_MAXK], sd[STAB_MAXK];
    __shared__ FitShared sh;
    __shared__ int s_last;
    __shared__ unsigned long long s_keys[2];
    const StreamDev &D = S[blockIdx.x];
    StreamState *st = D.st;
    const int tid = threadIdx.x, parts = gridDim.y, nwarps = blockDim.x >> 5;
    const long long t = io.src ? io.t : st->t - D.lag;   // transition tracked by this step
    if (!io.src && t < 0) {   // a batch's first step: no transition yet (nothing to record)
        if (threadIdx.x == 0 && blockIdx.y == 0) st->out_frame[st->t & 1] = -1;
        return;
    }
    int n = io.src ? *io.n : (t >= 1 ? st->n_pairs : 0);
    n = min(max(n, 0), D.K);
    const float2 *src = io.src ? io.src : D.pair_src;
    const float2 *dst = io.src ? io.dst : D.pair_dst;
    const int model = io.src ? io.model : D.model;
    const bool hybrid = model == STAB_HYBRID;
    const bool decide = hybrid && t >= 1 && (t - 1) % D.dwell == 0;
    int rigid = hybrid ? st->hyb_rigid : (model == STAB_RIGID);
    const float cx = __fmul_rn(0.5f, (float)(D.w - 1)), cy = __fmul_rn(0.5f, (float)(D.h - 1));
    for (int i = tid; i < n; i += blockDim.x) {
        float2 a = src[i], b = dst[i];
        ss[i] = make_float2(__fsub_rn(a.x, cx), __fsub_rn(a.y, cy));
        sd[i] = make_float2(__fsub_rn(b.x, cx), __fsub_rn(b.y, cy));
    }
    __syncthreads();
    const bool fitting = t >= 1 && n >= max(2, D.min_fit);
    // models fitted: both (rigid first) on a decision transition, else the held one
    const int nm = decide ? 2 : 1;
    const Mod64 mn = mod64_of((unsigned)max(n, 2)), mn1 = mod64_of((unsigned)max(n - 1, 1));
    if (fitting) {
        const int g = blockIdx.y * nwarps + (tid >> 5), G = parts * nwarps;
        for (int mi = 0; mi < nm; ++mi) {
            const unsigned long long k = score_slice(ss, sd, n, decide ? 1 - mi : rigid, D, t, g, G, mn, mn1, sh.key);
            if (tid == 0) atomicMax(&st->fit_key[mi], k);
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&st->fit_ticket, 1) == parts - 1;
    }
    __syncthreads();
    if (!s_last) return;
    if (tid == 0) {
        __threadfence();
        s_keys[0] = atomicExch(&st->fit_key[0], 0ull);
        s_keys[1] = atomicExch(&st->fit_key[1], 0ull);
        st->fit_ticket = 0;
    }
    __syncthreads();
    stab_motion out;
    out.tx = out.ty = out.theta = out.log_scale = 0.f;
    out.inliers = 0;
    out.n_tracks = n;
    out.rms = 0.f;
    out.e_rigid = out.e_similarity = -1.f;
    out.flags = (!io.src && st->due) ? STAB_FLAG_DETECTED : 0;
    if (decide) out.flags |= STAB_FLAG_DECISION;
    FitRes res;
    res.ok = false;
    if (fitting) {
        if (decide) {
            const FitRes fr = refit(ss, sd, n, 1, D, t, s_keys[0], mn, mn1, sh);
            const FitRes fs = refit(ss, sd, n, 0, D, t, s_keys[1], mn, mn1, sh);
            if (fr.ok) out.e_rigid = fr.rms;
            if (fs.ok) out.e_similarity = fs.rms;
            if (fr.ok && fs.ok) rigid = fr.rms < fs.rms;
            else if (fr.ok || fs.ok) rigid = fr.ok;
            res = rigid ? fr : fs;
        } else {
            res = refit(ss, sd, n, rigid, D, t, s_keys[0], mn, mn1, sh);
            if (res.ok) (rigid ? out.e_rigid : out.e_similarity) = res.rms;
        }
    }
    if (res.ok) {
        out.tx = res.tx; out.ty = res.ty; out.theta = res.th; out.log_scale = res.ls;
        out.inliers = res.inliers;
        out.rms = res.rms;
    } else if (t >= 1) {
        out.flags |= STAB_FLAG_SKIPPED;
    }
    if (rigid) out.flags |= STAB_FLAG_RIGID;
    if (tid == 0) {
        if (decide) st->hyb_rigid = rigid;
        if (io.out) *io.out = out;
        if (!io.src) D.mring[t % STAB_CRING] = out;
    }
    if (tid < 32 && !io.src && streaming) {
        __syncwarp();
        // this step's slot; the next step's warp composes frame u with it
        const int slot = (int)(st->t & 1);
        const int u = smooth_step(D.mring, D.cring, t, D.W, D.w, D.h, D.zoom, D.Minv + 8 * slot);
        if (tid == 0) st->out_frame[slot] = u;
    }
}

// ---------------------------------------------------------------------------
// 6-DOF affine fit (Eq. 7-8): three-point hypotheses, the same scoring, and
// the least squares of Eq. 7 on the winner's inliers.
__device__ __forceinline__ void sample_triple(unsigned long long seed, long long t, int h, int n, int &i, int &j,
                                              int &k)
{
    unsigned long long base = seed ^ ((unsigned long long)(unsigned)t << 32) ^ ((unsigned long long)(unsigned)h << 8);
    sample_pair(seed, t, h, mod64_of((unsigned)n), mod64_of((unsigned)(n - 1)), i, j);
    const int lo = min(i, j), hi = max(i, j);
    int c = (int)(splitmix64(base ^ 2ull) % (unsigned long long)(n - 2));
    if (c >= lo) ++c;
    if (c >= hi) ++c;
    k = c;
}

// A [u1 u2] = [v1 v2] through three pairs; m = (a00, a01, a10, a11, tx, ty).
__device__ __forceinline__ bool three_point(float2 si, float2 sj, float2 sk, float2 di, float2 dj, float2 dk, float m[6])
{
    const float u1x = __fsub_rn(sj.x, si.x), u1y = __fsub_rn(sj.y, si.y);
    const float u2x = __fsub_rn(sk.x, si.x), u2y = __fsub_rn(sk.y, si.y);
    const float v1x = __fsub_rn(dj.x, di.x), v1y = __fsub_rn(dj.y, di.y);
    const float v2x = __fsub_rn(dk.x, di.x), v2y = __fsub_rn(dk.y, di.y);
    const float det = __fmaf_rn(u1x, u2y, -__fmul_rn(u1y, u2x));
    if (!(fabsf(det) >= 1.0f)) return false;
    m[0] = __fdiv_rn(__fmaf_rn(v1x, u2y, -__fmul_rn(v2x, u1y)), det);
    m[1] = __fdiv_rn(__fmaf_rn(v2x, u1x, -__fmul_rn(v1x, u2x)), det);
    m[2] = __fdiv_rn(__fmaf_rn(v1y, u2y, -__fmul_rn(v2y, u1y)), det);
    m[3] = __fdiv_rn(__fmaf_rn(v2y, u1x, -__fmul_rn(v1y, u2x)), det);
    m[4] = __fsub_rn(di.x, __fmaf_rn(m[0], si.x, __fmul_rn(m[1], si.y)));
    m[5] = __fsub_rn(di.y, __fmaf_rn(m[2], si.x, __fmul_rn(m[3], si.y)));
    return true;
}

__device__ __forceinline__ bool is_inlier_affine(const float m[6], float2 s, float2 d, float tau2)
{
    const float px = __fmaf_rn(m[0], s.x, __fmaf_rn(m[1], s.y, m[4]));
    const float py = __fmaf_rn(m[2], s.x, __fmaf_rn(m[3], s.y, m[5]));
    const float ex = __fsub_rn(d.x, px), ey = __fsub_rn(d.y, py);
    return __fmaf_rn(ex, ex, __fmul_rn(ey, ey)) < tau2;
}

__global__ void __launch_bounds__(512) k_fit_affine(const StreamDev *__restrict__ S, AffineIO io)
{
    __shared__ float2 ss[STAB_MAXK], sd[STAB_MAXK];
    __shared__ int wbs[16], wbh[16], s_best, s_bh;
    __shared__ float red[16][8];
    const StreamDev &D = S[0];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
    const long long t = io.t;
    const int n = min(max(*io.n, 0), D.K);
    const float cx = __fmul_rn(0.5f, (float)(D.w - 1)), cy = __fmul_rn(0.5f, (float)(D.h - 1));
    for (int i = tid; i < n; i += blockDim.x) {
        const float2 a = io.src[i], b = io.dst[i];
        ss[i] = make_float2(__fsub_rn(a.x, cx), __fsub_rn(a.y, cy));
        sd[i] = make_float2(__fsub_rn(b.x, cx), __fsub_rn(b.y, cy));
    }
    __syncthreads();
    stab_affine out;
    out.a00 = 1.f; out.a01 = 0.f; out.a10 = 0.f; out.a11 = 1.f; out.tx = 0.f; out.ty = 0.f;
    out.inliers = 0; out.n_tracks = n; out.rms = 0.f; out.flags = STAB_FLAG_SKIPPED;
    if (n >= max(3, D.min_fit)) {
        int best = -1, bh = 0x7fffffff;
        for (int hh = wid; hh < D.H; hh += nwarps) {
            int i, j, k;
            sample_triple(D.seed, t, hh, n, i, j, k);
            float m[6];
            int cnt = -1;
            if (three_point(ss[i], ss[j], ss[k], sd[i], sd[j], sd[k], m)) {
                int c = 0;
                for (int q = lane; q < n; q += 32) c += is_inlier_affine(m, ss[q], sd[q], D.tau2);
                cnt = __reduce_add_sync(0xffffffffu, c);
            }
            if (cnt > best) { best = cnt; bh = hh; }
        }
        if (lane == 0) { wbs[wid] = best; wbh[wid] = bh; }
        __syncthreads();
        if (tid == 0) {
            int b = -1, h = 0x7fffffff;
            for (int q = 0; q < nwarps; ++q)
                if (wbs[q] > b || (wbs[q] == b && wbh[q] < h)) { b = wbs[q]; h = wbh[q]; }
            s_best = b; s_bh = h;
        }
        __syncthreads();
        if (s_best >= 3) {
            int i, j, k;
            sample_triple(D.seed, t, s_bh, n, i, j, k);
            float m[6];
            three_point(ss[i], ss[j], ss[k], sd[i], sd[j], sd[k], m);
            float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int q = tid; q < n; q += blockDim.x)
                if (is_inlier_affine(m, ss[q], sd[q], D.tau2)) {
                    v[0] += 1.f; v[1] += ss[q].x; v[2] += ss[q].y; v[3] += sd[q].x; v[4] += sd[q].y;
                }
            block_sum<8>(v, red);
            const float ni = v[0];
            const float msx = v[1] / ni, msy = v[2] / ni, mdx = v[3] / ni, mdy = v[4] / ni;
            float u[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // Sxx00, Sxx01, Sxx11, Syx00, Syx01, Syx10, Syx11
            for (int q = tid; q < n; q += blockDim.x)
                if (is_inlier_affine(m, ss[q], sd[q], D.tau2)) {
                    const float x0 = ss[q].x - msx, x1 = ss[q].y - msy, y0 = sd[q].x - mdx, y1 = sd[q].y - mdy;
                    u[0] += x0 * x0; u[1] += x0 * x1; u[2] += x1 * x1;
                    u[3] += y0 * x0; u[4] += y0 * x1; u[5] += y1 * x0; u[6] += y1 * x1;
                }
            block_sum<8>(u, red);
            const float det = u[0] * u[2] - u[1] * u[1];
            if (det > 0.f) {
                const float i00 = u[2] / det, i01 = -u[1] / det, i11 = u[0] / det;
                const float a00 = u[3] * i00 + u[4] * i01, a01 = u[3] * i01 + u[4] * i11;
                const float a10 = u[5] * i00 + u[6] * i01, a11 = u[5] * i01 + u[6] * i11;
                const float tx = mdx - (a00 * msx + a01 * msy), ty = mdy - (a10 * msx + a11 * msy);
                float e[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int q = tid; q < n; q += blockDim.x)
                    if (is_inlier_affine(m, ss[q], sd[q], D.tau2)) {
                        const float px = a00 * ss[q].x + a01 * ss[q].y + tx, py = a10 * ss[q].x + a11 * ss[q].y + ty;
                        e[0] += (sd[q].x - px) * (sd[q].x - px) + (sd[q].y - py) * (sd[q].y - py);
                    }
                block_sum<8>(e, red);
                out.a00 = a00; out.a01 = a01; out.a10 = a10; out.a11 = a11; out.tx = tx; out.ty = ty;
                out.inliers = (int)ni;
                out.rms = sqrtf(e[0] / ni);
                out.flags = 0;
            }
        }
    }
    if (tid == 0) *io.out = out;
}

// Offline smoothing in three launches (no scratch beyond the outputs):
// (1) trajectory C into the Minv buffer, (2) m' from C, (3) Minv from m'.
__global__ void k_smooth_c(const stab_motion *m, int T, float *Cbuf)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float4 C = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t = 0; t < T; ++t) {
        C = add4(C, mot4(m[t]));
        Cbuf[6 * t + 0] = C.x; Cbuf[6 * t + 1] = C.y; Cbuf[6 * t + 2] = C.z; Cbuf[6 * t + 3] = C.w;
    }
}

__global__ void k_smooth_mp(const stab_motion *m, int T, int W, const float *Cbuf, float *mprime)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        int lo = t - (W - 1) / 2, hi = t + W / 2;
        if (lo < 0) lo = 0;
        if (hi > T - 1) hi = T - 1;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = lo; k <= hi; ++k) acc = add4(acc, make_float4(Cbuf[6 * k], Cbuf[6 * k + 1], Cbuf[6 * k + 2], Cbuf[6 * k + 3]));
        const float cnt = (float)(hi - lo + 1);
        const float4 Sm = make_float4(__fdiv_rn(acc.x, cnt), __fdiv_rn(acc.y, cnt), __fdiv_rn(acc.z, cnt),
                                      __fdiv_rn(acc.w, cnt));
        const float4 Ct = make_float4(Cbuf[6 * t], Cbuf[6 * t + 1], Cbuf[6 * t + 2], Cbuf[6 * t + 3]);
        const float4 mp = corrected(mot4(m[t]), Sm, Ct);
        mprime[4 * t + 0] = mp.x; mprime[4 * t + 1] = mp.y; mprime[4 * t + 2] = mp.z; mprime[4 * t + 3] = mp.w;
    }
}

__global__ void k_smooth_minv(const float *mprime, int T, int w, int h, float zoom, float *Minv)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        inverse_warp(make_float4(mprime[4 * t], mprime[4 * t + 1], mprime[4 * t + 2], mprime[4 * t + 3]), w, h,
                     zoom, Minv + 6 * t);
}

__global__ void k_smooth_push(const StreamDev *__restrict__ S, long long t, const stab_motion *m, float *Minv,
                              int *ready)
{
    const StreamDev &D = S[0];   // one warp
    if (threadIdx.x == 0) D.mring[t % STAB_CRING] = *m;
    __syncwarp();
    float M[6];
    const int u = smooth_step(D.mring, D.cring, t, D.W, D.w, D.h, D.zoom, M);
    if (threadIdx.x == 0) {
        if (u >= 0)
            for (int k = 0; k < 6; ++k) Minv[k] = M[k];
        *ready = u;
    }
}

__global__ void k_advance(const StreamDev *__restrict__ S, int n)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) S[s].st->t += 1;
}

}  // namespace

void launch_compact(const Launch &L, const StreamDev *S, int n, CompactIO io)
{
    k_compact<<<n, 1024, 0, L.stream>>>(S, io);
}

void launch_fit(const Launch &L, const StreamDev *S, int n, FitIO io, int streaming, int hmax)
{
    // one hypothesis or more per scoring warp (16 per CTA), at most 8 CTAs per stream
    const int parts = hmax <= 16 ? 1 : hmax >= 8 * 16 ? 8 : (hmax + 15) / 16;
    k_fit<<<dim3(n, parts), 512, 0, L.stream>>>(S, io, streaming);
}

void launch_fit_affine(const Launch &L, const StreamDev *S, AffineIO io)
{
    k_fit_affine<<<1, 512, 0, L.stream>>>(S, io);
}

void launch_smooth_offline(const Launch &L, const stab_motion *m, int T, int W, int w, int h, float zoom,
                           float *mprime, float *Minv)
{
    k_smooth_c<<<1, 32, 0, L.stream>>>(m, T, Minv);
    k_smooth_mp<<<(T + 255) / 256, 256, 0, L.stream>>>(m, T, W, Minv, mprime);
    k_smooth_minv<<<(T + 255) / 256, 256, 0, L.stream>>>(mprime, T, w, h, zoom, Minv);
}

void launch_smooth_push(const Launch &L, const StreamDev *S, long long t, const stab_motion *m, float *Minv,
                        int *ready)
{
    k_smooth_push<<<1, 32, 0, L.stream>>>(S, t, m, Minv, ready);
}

void launch_advance(const Launch &L, const StreamDev *S, int n)
{
    k_advance<<<(n + 63) / 64, 64, 0, L.stream>>>(S, n);
}

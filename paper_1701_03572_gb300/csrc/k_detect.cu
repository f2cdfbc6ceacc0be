// k_detect.cu -- Shi-Tomasi corners on the reduced region of interest
// (Sec. 3.1, Eq. 2) and exact top-K selection.
//
//  k_begin     per stream: frame index, whether detection is due, counters.
//  k_response  vertical strips of the ROI (a thread walks 4 columns down 20
//              rows): Sobel 3x3 -> integer tensor over a 3x3 box -> FP32 min
//              eigenvalue -> 3x3 non-maximum suppression.  Survivors are
//              appended as 64-bit keys (score bits << 32 | ~raster index), so
//              that "larger key" means "higher score, then lower index", and
//              counted in a 4096-bin histogram of the score's top 12 bits.  The
//              last strip of a stream to finish turns the histogram into the
//              bin where the K-th key lives.
//  k_filter    keeps keys at or above that bin and above q * max.
//  k_select    one CTA per stream: radix select of the K-th largest key in
//              shared memory, compaction, bitonic sort, points out.
// The score is computed in the same FP32 operation sequence the oracle uses
// (2 det / (tr + sqrt(disc)) from exact int64 terms), so rankings are exact.
#include "kernels.cuh"

#define FCHUNK 2048

namespace {

// Round-to-nearest-even FP32 value of an integer 0 <= v < 2^57, without the
// 64-bit conversion instruction (GB300 runs it on its narrow FP64 pipe): v >> s
// keeps v's 26 leading bits and every bit shifted out is ORed into the lowest
// (sticky) bit, so rounding those 26 bits to 24 picks the same significand as
// rounding v; the scale by 2^s is then exact.
__device__ __forceinline__ float u57_to_f32(unsigned long long v)
{
    const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    const int s = hi ? 38 - __clz(hi) : 0;   // hi < 2^25: s <= 31
    const unsigned z = __funnelshift_r(lo, hi, s) | (unsigned)((lo & ((1u << s) - 1u)) != 0u);
    return __fmul_rn(__uint2float_rn(z), __int_as_float((127 + s) << 23));
}

// a, c <= 9 (4 * 255)^2 < 2^24, so tr < 2^25 converts from 32 bits; det < 2^47
// and disc <= tr^2 < 2^50 are non-negative (the tensor is a sum of outer
// products) and exact in 64 bits.
__device__ __forceinline__ float lambda32(int a, int b, int c)
{
    const int tr = a + c;
    if (tr == 0) return 0.0f;
    const long long det = (long long)a * c - (long long)b * b;
    const int d = a - c;
    const long long disc = (long long)d * d + 4 * ((long long)b * b);
    const float num = __fmul_rn(2.0f, u57_to_f32((unsigned long long)det));
    const float den = __fadd_rn(__int2float_rn(tr), __fsqrt_rn(u57_to_f32((unsigned long long)disc)));
    return __fdiv_rn(num, den);
}

__global__ void k_begin(const StreamDev *__restrict__ S, int n, long long t_ov, int force_due)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const StreamDev &D = S[s];
    StreamState *st = D.st;
    long long t = t_ov >= 0 ? t_ov : st->t;
    st->t = t;
    const long long tb = t - D.lag;   // transition tracked by this step: frames tb-1 -> tb
    int due;
    if (force_due) due = 1;
    else due = (tb >= 1) && (st->n_feat == 0 || ((tb - 1 + D.phase) % D.period) == 0 || st->n_feat < D.min_tracks);
    st->due = due;
    // detection-due count of this step (read by the detection kernels, which
    // return at once when it is 0); the other parity's count is cleared for
    // the next step
    if (due) atomicAdd(&S[0].st->n_due[t & 1], 1);
    if (s == 0) S[0].st->n_due[(t + 1) & 1] = 0;
    st->n_cand = 0;
    st->n_sel = 0;
    st->n_above = 0;
    st->lam_max = 0;
    st->blocks_done = 0;
    st->iters = 0;
    st->tpl = 0;
}

// One pixel row's bytes at columns x-1 .. x+4, clamped into the frame.  Inside
// the row they come from three aligned words (columns x-4 .. x+7), which the
// caller loads one row ahead (rs_words); near a border they are read singly.
struct RsWords { unsigned w0, w1, w2; };

__device__ __forceinline__ RsWords rs_words(const uint8_t *__restrict__ g, int pitch, int h, int x, int yy)
{
    const unsigned *q = reinterpret_cast<const unsigned *>(g + (size_t)clampi(yy, 0, h - 1) * pitch + x - 4);
    return RsWords{__ldg(q), __ldg(q + 1), __ldg(q + 2)};
}

__device__ __forceinline__ void rs_pixels(const uint8_t *__restrict__ g, int pitch, int w, int h, int x, int yy,
                                          bool fast, RsWords v, int (&p)[6])
{
    if (fast) {
        p[0] = v.w0 >> 24;
        p[1] = v.w1 & 255u; p[2] = (v.w1 >> 8) & 255u; p[3] = (v.w1 >> 16) & 255u; p[4] = v.w1 >> 24;
        p[5] = v.w2 & 255u;
    } else {
        const uint8_t *row = g + (size_t)clampi(yy, 0, h - 1) * pitch;
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = __ldg(row + clampi(x - 1 + k, 0, w - 1));
    }
}

// True when k_begin found no stream due for detection at this step.
__device__ __forceinline__ bool no_detection_due(const StreamDev *__restrict__ S)
{
    const StreamState *s0 = S[0].st;
    return __ldcg(&s0->n_due[s0->t & 1]) == 0;
}

// Candidates of a strip are collected in the warp's shared-memory buffer and
// appended to the stream's list with one global atomic per strip (a full
// buffer appends the warp's candidates directly).
constexpr int RS_CAP = 256;

// A compile-time slot index passed to the row step of k_response.
template <int I>
struct Slot { static constexpr int value = I; };

// Corner response (Eq. 2), NMS and candidate list as barrier-free vertical
// strips, each warp on its own: a warp owns a strip of 120 ROI columns and 20
// rows (drawn from an atomic ticket when the work list has one), a thread
// columns x .. x+3 of it, and walks its pixel rows once.  Per pixel row it forms the separable Sobel parts
// (horizontal difference and [1 2 1] smoothing) of its 4 columns and keeps two
// rows of them; three rows give gx, gy of the previous row, whose products are
// summed over 3 columns (the products of columns x-1 and x+4 come from the
// neighbouring lanes) and kept for two rows more; three such rows give the 3x3
// structure tensor and the score two rows back, and three score rows (the
// neighbours' outer scores again by shuffle) give the NMS of the row before.
// Lanes 0 and 31 of a warp compute their columns only for lanes 1 and 30 and
// emit nothing.  Integer sums are exact; the score is lambda32 of them.
__global__ void __launch_bounds__(STAB_RS_THREADS, 4) k_response(const StreamDev *__restrict__ S, WorkList wl, DetIO io)
{
    __shared__ unsigned long long s_keys[STAB_RS_THREADS / 32][RS_CAP];
    if (no_detection_due(S)) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    unsigned long long *wkeys = s_keys[wp];
    const int nwarps = gridDim.x * (STAB_RS_THREADS / 32);
    int item = blockIdx.x * (STAB_RS_THREADS / 32) + wp, tk = 0;
    if (wl.ctr) item = __shfl_sync(0xffffffffu, lane == 0 ? (int)atomicAdd(wl.ctr, 1u) : 0, 0);
    for (; item < wl.total; item = wl.ctr ? __shfl_sync(0xffffffffu, tk, 0) : item + nwarps) {
        if (wl.ctr && lane == 0) tk = (int)atomicAdd(wl.ctr, 1u);   // drawn now, used after this strip
        const int s = wl_stream(wl, item);
        const StreamDev &D = S[s];
        StreamState *st = D.st;
        if (!st->due) continue;
        const int local = item - __ldg(&wl.prefix[s]);
        const int ntiles = __ldg(&wl.prefix[s + 1]) - __ldg(&wl.prefix[s]);
        const uint8_t *g;
        int pitch;
        if (io.gray) { g = io.gray; pitch = io.pitch; }
        else { g = D.u8[stab_pslot(st->t - D.lag - 1)][0]; pitch = D.lp[0]; }
        const int w = D.w, h = D.h;
        const int rx1 = D.roi_x1, ry1 = D.roi_y1;
        const int ngx = (rx1 - D.roi_x0 + STAB_RS_COLS - 1) / STAB_RS_COLS;
        const int x = D.roi_x0 + (local % ngx) * STAB_RS_COLS + 4 * (lane - 1);
        const bool owner = lane >= 1 && lane <= 30;   // lanes 0 and 31 only supply neighbours
        const int y0 = D.roi_y0 + (local / ngx) * STAB_RS_ROWS;
        const int nrows = min(STAB_RS_ROWS, ry1 - y0);
        const bool fast = x >= 4 && x + 8 <= w && ((x | pitch) & 3) == 0 && (reinterpret_cast<uintptr_t>(g) & 3) == 0;
        int wn = 0;   // candidates in the warp's buffer (the same in every lane)
        // Row windows of period 3, in slots rotated by the unrolled loop (no
        // register moves): Sobel parts d, sm of pixel rows, tensor row sums ha, hb,
        // hc, scores l (own columns x .. x+3; the scores also hold columns x-1
        // (index 0) and x+4 (index 5)).
        int d[3][4] = {}, sm[3][4] = {}, ha[3][4] = {}, hb[3][4] = {}, hc[3][4] = {};
        float l[3][6] = {};
        unsigned lmax = 0;
        const int nk = nrows + 6, nk3 = ((nk + 2) / 3) * 3;   // rows past nk emit nothing
        RsWords nxt = fast ? rs_words(g, pitch, h, x, y0 - 3) : RsWords{0u, 0u, 0u};
        // Row k: pixel row py = y0 - 3 + k enters in slot N (the rows before it are
        // in slots P, then O).
        auto row = [&](auto cn, auto cp, auto co, int k) {
            constexpr int N = decltype(cn)::value, P = decltype(cp)::value, O = decltype(co)::value;
            const int py = y0 - 3 + k;
            const RsWords cur = nxt;
            if (fast && k + 1 < nk3) nxt = rs_words(g, pitch, h, x, py + 1);   // next row in flight
            int p[6];
            rs_pixels(g, pitch, w, h, x, py, fast, cur, p);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                d[N][j] = p[j + 2] - p[j];
                sm[N][j] = p[j] + 2 * p[j + 1] + p[j + 2];
            }
            // gx, gy of row py-1 at columns x .. x+3 (index 1 .. 4); the products of
            // columns x-1 and x+4 come from the neighbouring lanes.  Only rows whose
            // tensor sums reach a score that an NMS reads (k >= 2) are formed, and only
            // scores that an NMS reads (rows k = 4 .. nk-1) are computed (k is the same
            // in every lane).
            if (k >= 2 && k < nk) {
                int A[6], B[6], C[6];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int gx = d[O][j] + 2 * d[P][j] + d[N][j], gy = sm[N][j] - sm[O][j];
                    A[j + 1] = gx * gx; B[j + 1] = gx * gy; C[j + 1] = gy * gy;
                }
                A[0] = __shfl_up_sync(0xffffffffu, A[4], 1); A[5] = __shfl_down_sync(0xffffffffu, A[1], 1);
                B[0] = __shfl_up_sync(0xffffffffu, B[4], 1); B[5] = __shfl_down_sync(0xffffffffu, B[1], 1);
                C[0] = __shfl_up_sync(0xffffffffu, C[4], 1); C[5] = __shfl_down_sync(0xffffffffu, C[1], 1);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ha[N][i] = A[i] + A[i + 1] + A[i + 2];
                    hb[N][i] = B[i] + B[i + 1] + B[i + 2];
                    hc[N][i] = C[i] + C[i + 1] + C[i + 2];
                }
            }
            // score of row py-2 at columns x .. x+3, and of x-1, x+4 from the neighbours
            if (k >= 4 && k < nk) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    l[N][i + 1] = lambda32(ha[O][i] + ha[P][i] + ha[N][i], hb[O][i] + hb[P][i] + hb[N][i],
                                           hc[O][i] + hc[P][i] + hc[N][i]);
                l[N][0] = __shfl_up_sync(0xffffffffu, l[N][4], 1);
                l[N][5] = __shfl_down_sync(0xffffffffu, l[N][1], 1);
            }
            // NMS of row py-3 (scores l[O] = row py-4, l[P] = py-3, l[N] = py-2)
            unsigned long long keys[2];
            int nk_ = 0;
            const int y = py - 3;
            if (k >= 6 && k < nk) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (owner && x + c < rx1) {
                        const float v = l[P][c + 1];
                        lmax = max(lmax, __float_as_uint(v));
                        // strict maximum over the 3x3 neighbourhood; a tie goes to the lower raster index
                        bool keep = v > 0.0f && v > l[O][c] && v > l[O][c + 1] && v > l[O][c + 2] && v > l[P][c];
                        keep = keep && v >= l[P][c + 2] && v >= l[N][c] && v >= l[N][c + 1] && v >= l[N][c + 2];
                        if (keep && nk_ < 2) {
                            const unsigned idx = (unsigned)(y * w + x + c);
                            keys[nk_++] = ((unsigned long long)__float_as_uint(v) << 32) |
                                          (unsigned long long)(0xFFFFFFFFu - idx);
                        }
                    }
                }
            }
            // warp-aggregated append of this row's candidates to the warp's buffer
            if (__any_sync(0xffffffffu, nk_ > 0)) {
                int incl = nk_;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                int base = wn;
                const bool full = wn + tot > RS_CAP;
                if (full) {   // this row's candidates go straight out
                    if (lane == 31) base = atomicAdd(&st->n_cand, tot);
                    base = __shfl_sync(0xffffffffu, base, 31);
                } else {
                    wn += tot;
                }
                const int pos = base + incl - nk_;
                for (int q = 0; q < nk_; ++q) {
                    if (!full) wkeys[pos + q] = keys[q];
                    else {
                        if (pos + q < D.cand_cap) D.cand[pos + q] = keys[q];
                        else set_err(st, STAB_ERR_CAPACITY);
                        atomicAdd(&D.hist[(unsigned)(keys[q] >> (32 + STAB_HSHIFT))], 1u);
                    }
                }
            }
        };
#pragma unroll 1
        for (int k = 0; k < nk3; k += 3) {
            row(Slot<0>{}, Slot<2>{}, Slot<1>{}, k);
            row(Slot<1>{}, Slot<0>{}, Slot<2>{}, k + 1);
            row(Slot<2>{}, Slot<1>{}, Slot<0>{}, k + 2);
        }
        // the strip's max score and its buffered candidates go out with one atomic each
        for (int o = 16; o; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        __syncwarp();   // the buffer's entries are visible to the whole warp
        int base = 0;
        if (lane == 0 && wn) base = atomicAdd(&st->n_cand, wn);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int i = lane; i < wn; i += 32) {
            const unsigned long long key = wkeys[i];
            if (base + i < D.cand_cap) D.cand[base + i] = key;
            else set_err(st, STAB_ERR_CAPACITY);
            atomicAdd(&D.hist[(unsigned)(key >> (32 + STAB_HSHIFT))], 1u);
        }
        __syncwarp();   // the buffer is refilled by the next strip
        int last = 0;
        if (lane == 0) {
            atomicMax(&st->lam_max, lmax);
            __threadfence();
            last = atomicAdd(&st->blocks_done, 1) == ntiles - 1;
        }
        if (__shfl_sync(0xffffffffu, last, 0)) {
            // This is the stream's last strip: every append and histogram count is
            // visible (they were made before each strip's fence and ticket).
            __threadfence();
            const unsigned lm = __ldcg(&st->lam_max);
            const float thr = __fmul_rn(D.quality, __uint_as_float(lm));
            const unsigned thr_bits = __float_as_uint(thr), tbin = thr_bits >> STAB_HSHIFT;
            // lane i owns bins [4095 - 128 i - 127, 4095 - 128 i], highest first; the
            // K-th key lies in the first bin (from the top) where the count reaches K.
            // A lane reads its bins as 16-byte vectors, eight vectors in flight at a
            // time, so the cut costs a few L2 round trips rather than one per bin.
            constexpr int BPL = STAB_HBINS / 32, VPL = BPL / 4, VB = 8;
            const int lo = STAB_HBINS - BPL * (lane + 1);   // lowest bin of the lane, 16-byte aligned
            const uint4 *hv = reinterpret_cast<const uint4 *>(D.hist + lo);
            const int tb = (int)tbin;
            unsigned cnt = 0;
            for (int v0 = 0; v0 < VPL; v0 += VB) {
                uint4 q[VB];
#pragma unroll
                for (int v = 0; v < VB; ++v) q[v] = __ldcg(hv + v0 + v);
#pragma unroll
                for (int v = 0; v < VB; ++v) {
                    const int b = lo + 4 * (v0 + v);   // bins b .. b+3
                    cnt += (b >= tb ? q[v].x : 0u) + (b + 1 >= tb ? q[v].y : 0u) + (b + 2 >= tb ? q[v].z : 0u) +
                           (b + 3 >= tb ? q[v].w : 0u);
                }
            }
            unsigned incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned K = (unsigned)D.K, excl = incl - cnt;
            unsigned bin = tbin;
            if (excl < K && K <= incl) {   // at most one lane: walk its bins from the top
                unsigned cum = excl;
                bool found = false;
                for (int v0 = VPL - VB; v0 >= 0 && !found; v0 -= VB) {
                    uint4 q[VB];
#pragma unroll
                    for (int v = 0; v < VB; ++v) q[v] = __ldcg(hv + v0 + v);
#pragma unroll
                    for (int v = VB - 1; v >= 0; --v) {
                        const int b = lo + 4 * (v0 + v);
                        const unsigned c4[4] = {q[v].x, q[v].y, q[v].z, q[v].w};
#pragma unroll
                        for (int e = 3; e >= 0; --e) {
                            if (!found && b + e >= tb) {
                                cum += c4[e];
                                if (cum >= K) { bin = (unsigned)(b + e); found = true; }
                            }
                        }
                    }
                }
            }
            const unsigned who = __ballot_sync(0xffffffffu, excl < K && K <= incl);
            if (who) bin = __shfl_sync(0xffffffffu, bin, __ffs(who) - 1);
            if (lane == 0) {
                st->bin_lo = bin > tbin ? bin : tbin;
                st->thr_bits = thr_bits;
            }
        }
    }
    // every warp has drawn a ticket past the end; the last to finish resets the list
    if (wl.ctr && lane == 0 && atomicAdd(wl.ctr + 1, 1u) == (unsigned)(nwarps - 1)) {
        atomicExch(wl.ctr, 0u);
        atomicExch(wl.ctr + 1, 0u);
    }
}

__global__ void __launch_bounds__(256) k_filter(const StreamDev *__restrict__ S, WorkList wl)
{
    if (no_detection_due(S)) return;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int item = blockIdx.x; item < wl.total; item += gridDim.x) {
        const int s = wl_stream(wl, item);
        const StreamDev &D = S[s];
        StreamState *st = D.st;
        if (!st->due) continue;
        const int c0 = (item - __ldg(&wl.prefix[s])) * FCHUNK;
        const int nc = min(st->n_cand, D.cand_cap);
        if (c0 >= nc) continue;
        const int end = min(c0 + FCHUNK, nc);
        const unsigned bin_lo = st->bin_lo, thr = st->thr_bits;
        for (int b0 = c0; b0 < end; b0 += blockDim.x) {
            int i = b0 + tid;
            unsigned long long key = 0;
            bool pass = false, above = false;
            if (i < end) {
                key = D.cand[i];
                unsigned lb = (unsigned)(key >> 32);
                above = lb > thr;
                pass = above && (lb >> STAB_HSHIFT) >= bin_lo;
            }
            unsigned m = __ballot_sync(0xffffffffu, pass);
            unsigned ma = __ballot_sync(0xffffffffu, above);
            int base = 0;
            if (lane == 0 && ma) atomicAdd(&st->n_above, __popc(ma));
            if (lane == 0 && m) base = atomicAdd(&st->n_sel, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (pass) D.sel[base + __popc(m & ((1u << lane) - 1u))] = key;
        }
    }
}

__global__ void __launch_bounds__(1024) k_select(const StreamDev *__restrict__ S, DetIO io)
{
    extern __shared__ unsigned long long skeys[];
    __shared__ unsigned long long sout[STAB_MAXK];
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix, s_mask;
    __shared__ int s_kk, s_cnt;
    const StreamDev &D = S[blockIdx.x];
    StreamState *st = D.st;
    if (!st->due) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const int n = st->n_sel;
    const int Kp = min(D.K, n);
    const unsigned long long *keys = D.sel;
    if (n <= STAB_SEL_SMEM) {
        for (int i = tid; i < n; i += blockDim.x) skeys[i] = D.sel[i];
        keys = skeys;
    }
    if (tid == 0) { s_prefix = 0; s_mask = 0; s_kk = Kp; s_cnt = 0; }
    __syncthreads();
    if (Kp < n) {
        for (int shift = 56; shift >= 0; shift -= 8) {
            if (tid < 256) hist[tid] = 0;
            __syncthreads();
            const unsigned long long pre = s_prefix, msk = s_mask;
            for (int i = tid; i < n; i += blockDim.x) {
                unsigned long long k = keys[i];
                if ((k & msk) == pre) atomicAdd(&hist[(unsigned)(k >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (tid < 32) {
                unsigned loc = 0;
                for (int j = 0; j < 8; ++j) loc += hist[255 - 8 * lane - j];
                unsigned incl = loc;
                for (int o = 1; o < 32; o <<= 1) {
                    unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                unsigned excl = incl - loc, kk = (unsigned)s_kk;
                if (excl < kk && kk <= incl) {
                    for (int j = 0; j < 8; ++j) {
                        unsigned d = 255 - 8 * lane - j, c = hist[d];
                        if (kk <= excl + c) {
                            s_prefix = pre | ((unsigned long long)d << shift);
                            s_mask = msk | (255ull << shift);
                            s_kk = (int)(kk - excl);
                            break;
                        }
                        excl += c;
                    }
                }
            }
            __syncthreads();
        }
    }
    const unsigned long long kth = (Kp < n) ? s_prefix : 0ull;
    for (int i = tid; i < n; i += blockDim.x) {
        unsigned long long k = keys[i];
        if (k >= kth) {
            int p = atomicAdd(&s_cnt, 1);
            if (p < STAB_MAXK) sout[p] = k;
        }
    }
    __syncthreads();
    if (tid == 0 && s_cnt != Kp) set_err(st, STAB_ERR_CAPACITY);
    int P = 1;
    while (P < Kp) P <<= 1;
    for (int i = Kp + tid; i < P; i += blockDim.x) sout[i] = 0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long a = sout[i], b = sout[ixj];
                    bool desc = (i & k) == 0;
                    if (desc ? (a < b) : (a > b)) { sout[i] = b; sout[ixj] = a; }
                }
            }
            __syncthreads();
        }
    for (int i = tid; i < Kp; i += blockDim.x) {
        unsigned long long k = sout[i];
        unsigned idx = 0xFFFFFFFFu - (unsigned)(k & 0xFFFFFFFFull);
        float2 p = make_float2((float)(idx % (unsigned)D.w), (float)(idx / (unsigned)D.w));
        float lam = __uint_as_float((unsigned)(k >> 32));
        D.feat[i] = p;
        D.det_lam[i] = lam;
        if (io.pts_out) io.pts_out[i] = p;
        if (io.lam_out) io.lam_out[i] = lam;
    }
    if (tid == 0) {
        st->n_feat = Kp;
        st->n_det = Kp;
        if (io.n_out) *io.n_out = Kp;
        if (io.ncand_out) *io.ncand_out = st->n_above;
    }
    for (int b = tid; b < STAB_HBINS; b += blockDim.x) D.hist[b] = 0u;
    (void)lane;
}

}  // namespace

void launch_begin(const Launch &L, const StreamDev *S, int n, long long t_ov, int force_due)
{
    k_begin<<<(n + 63) / 64, 64, 0, L.stream>>>(S, n, t_ov, force_due);
}

static int occ_response()
{
    static DevCache c;
    return c.get([] {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_response, STAB_RS_THREADS, 0) != cudaSuccess ||
            occ < 1)
            occ = 1;
        return occ;
    });
}

// k_select's dynamic shared memory exceeds the default limit: the attribute is
// set once on every device the selection runs on.
static void select_attr()
{
    static DevCache c;
    c.get([] {
        cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, STAB_SEL_SMEM * 8);
        return 1;
    });
}

void warm_detect()
{
    occ_response();
    select_attr();
}

void launch_response(const Launch &L, const StreamDev *S, WorkList wl, DetIO io)
{
    const int blocks = (wl.total + STAB_RS_THREADS / 32 - 1) / (STAB_RS_THREADS / 32);   // a warp per strip
    k_response<<<grid_for(L, blocks, occ_response()), STAB_RS_THREADS, 0, L.stream>>>(S, wl, io);
}

void launch_filter(const Launch &L, const StreamDev *S, WorkList wl)
{
    k_filter<<<grid_for(L, wl.total, 4), 256, 0, L.stream>>>(S, wl);
}

void launch_select(const Launch &L, const StreamDev *S, int n, DetIO io)
{
    select_attr();
    k_select<<<n, 1024, STAB_SEL_SMEM * 8, L.stream>>>(S, io);
}

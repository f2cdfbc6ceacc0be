// k_detect.cu -- Shi-Tomasi corners on the reduced region of interest
// (Sec. 3.1, Eq. 2) and exact top-K selection.
//
//  k_begin     per stream: frame index, whether detection is due, counters.
//  k_response  64 x 16 ROI tiles staged in shared memory with a 3-px halo:
//              Sobel 3x3 -> integer tensor over a 3x3 box -> FP32 min
//              eigenvalue -> 3x3 non-maximum suppression.  Survivors are
//              appended as 64-bit keys (score bits << 32 | ~raster index), so
//              that "larger key" means "higher score, then lower index", and
//              counted in a 4096-bin histogram of the score's top 12 bits.  The
//              last tile of a stream to finish turns the histogram into the
//              bin where the K-th key lives.
//  k_filter    keeps keys at or above that bin and above q * max.
//  k_select    one CTA per stream: radix select of the K-th largest key in
//              shared memory, compaction, bitonic sort, points out.
// The score is computed in the same FP32 operation sequence the oracle uses
// (2 det / (tr + sqrt(disc)) from exact int64 terms), so rankings are exact.
#include "kernels.cuh"

#define FCHUNK 2048

namespace {

__device__ __forceinline__ float lambda32(int a, int b, int c)
{
    long long tr = (long long)a + c;
    if (tr == 0) return 0.0f;
    long long det = (long long)a * c - (long long)b * b;
    long long d = (long long)a - c;
    long long disc = d * d + 4 * (long long)b * b;
    float num = __ll2float_rn(2 * det);
    float den = __fadd_rn(__ll2float_rn(tr), __fsqrt_rn(__ll2float_rn(disc)));
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
    int due;
    if (force_due) due = 1;
    else due = (t >= 1) && (st->n_feat == 0 || ((t - 1) % D.period) == 0 || st->n_feat < D.min_tracks);
    st->due = due;
    st->n_cand = 0;
    st->n_sel = 0;
    st->n_above = 0;
    st->lam_max = 0;
    st->blocks_done = 0;
    st->iters = 0;
    st->tpl = 0;
}

__global__ void __launch_bounds__(256) k_response(const StreamDev *__restrict__ S, WorkList wl, DetIO io)
{
    constexpr int TW = STAB_TW, TH = STAB_TH;
    constexpr int PW = TW + 6, PH = TH + 6;   // pixels
    constexpr int GW = TW + 4, GH = TH + 4;   // Sobel
    constexpr int LW = TW + 2, LH = TH + 2;   // scores (tile + NMS ring)
    __shared__ uint8_t spx[PH][PW + 2];
    __shared__ short sgx[GH][GW], sgy[GH][GW];
    __shared__ float slam[LH][LW];
    __shared__ unsigned smax;
    __shared__ int s_last;
    __shared__ unsigned s_cnt[256];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int item = blockIdx.x; item < wl.total; item += gridDim.x) {
        const int s = wl_stream(wl, item);
        const StreamDev &D = S[s];
        StreamState *st = D.st;
        if (!st->due) continue;
        const int local = item - __ldg(&wl.prefix[s]);
        const int ntiles = __ldg(&wl.prefix[s + 1]) - __ldg(&wl.prefix[s]);
        const uint8_t *g;
        int pitch;
        if (io.gray) { g = io.gray; pitch = io.pitch; }
        else { g = D.u8[(int)((st->t - 1) & 1)][0]; pitch = D.lp[0]; }
        const int w = D.w, h = D.h;
        const int rx1 = D.roi_x1, ry1 = D.roi_y1;
        const int tiles_x = (rx1 - D.roi_x0 + TW - 1) / TW;
        const int x0 = D.roi_x0 + (local % tiles_x) * TW, y0 = D.roi_y0 + (local / tiles_x) * TH;
        for (int i = tid; i < PH * PW; i += blockDim.x) {
            int r = i / PW, c = i - r * PW;
            spx[r][c] = __ldg(g + (size_t)clampi(y0 - 3 + r, 0, h - 1) * pitch + clampi(x0 - 3 + c, 0, w - 1));
        }
        if (tid == 0) smax = 0;
        __syncthreads();
        for (int i = tid; i < GH * GW; i += blockDim.x) {
            int r = i / GW, c = i - r * GW;
            int gx = (spx[r][c + 2] + 2 * spx[r + 1][c + 2] + spx[r + 2][c + 2]) -
                     (spx[r][c] + 2 * spx[r + 1][c] + spx[r + 2][c]);
            int gy = (spx[r + 2][c] + 2 * spx[r + 2][c + 1] + spx[r + 2][c + 2]) -
                     (spx[r][c] + 2 * spx[r][c + 1] + spx[r][c + 2]);
            sgx[r][c] = (short)gx;
            sgy[r][c] = (short)gy;
        }
        __syncthreads();
        for (int i = tid; i < LH * LW; i += blockDim.x) {
            int r = i / LW, c = i - r * LW;
            int a = 0, b = 0, cc = 0;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    int gx = sgx[r + dy][c + dx], gy = sgy[r + dy][c + dx];
                    a += gx * gx;
                    b += gx * gy;
                    cc += gy * gy;
                }
            slam[r][c] = lambda32(a, b, cc);
        }
        __syncthreads();
        // NMS on 4 consecutive pixels of one row
        const int row = tid >> 4, c4 = (tid & 15) * 4;
        const int y = y0 + row;
        unsigned long long keys[2];
        int nk = 0;
        unsigned lmax = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int x = x0 + c4 + k;
            if (x < rx1 && y < ry1) {
                int r = row + 1, c = c4 + k + 1;
                float v = slam[r][c];
                lmax = max(lmax, __float_as_uint(v));
                bool keep = v > 0.0f;
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (dx == 0 && dy == 0) continue;
                        float u = slam[r + dy][c + dx];
                        bool after = (dy > 0) || (dy == 0 && dx > 0);   // neighbour later in raster order
                        keep = keep && (v > u || (v == u && after));
                    }
                if (keep && nk < 2) {
                    unsigned idx = (unsigned)(y * w + x);
                    keys[nk++] = ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xFFFFFFFFu - idx);
                }
            }
        }
        // block max of the score
        for (int o = 16; o; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        if (lane == 0) atomicMax(&smax, lmax);
        // warp-aggregated append
        int incl = nk;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int tot = __shfl_sync(0xffffffffu, incl, 31);
        int base = 0;
        if (lane == 31 && tot) base = atomicAdd(&st->n_cand, tot);
        base = __shfl_sync(0xffffffffu, base, 31);
        int pos = base + incl - nk;
        for (int k = 0; k < nk; ++k) {
            if (pos + k < D.cand_cap) D.cand[pos + k] = keys[k];
            else set_err(st, STAB_ERR_CAPACITY);
            atomicAdd(&D.hist[(unsigned)(keys[k] >> (32 + STAB_HSHIFT))], 1u);
        }
        __syncthreads();
        if (tid == 0) {
            atomicMax(&st->lam_max, smax);
            __threadfence();
            int done = atomicAdd(&st->blocks_done, 1);
            s_last = (done == ntiles - 1);
        }
        __syncthreads();
        if (s_last) {
            // This is the stream's last tile: every append and histogram count is
            // visible (they were made before each tile's fence and ticket).
            __threadfence();
            unsigned lm = __ldcg(&st->lam_max);
            float thr = __fmul_rn(D.quality, __uint_as_float(lm));
            unsigned thr_bits = __float_as_uint(thr);
            unsigned tbin = thr_bits >> STAB_HSHIFT;
            // thread i owns bins [4095 - 16 i - 15, 4095 - 16 i], highest first
            unsigned cnt = 0;
            for (int j = 0; j < 16; ++j) {
                unsigned b = STAB_HBINS - 1 - 16 * tid - j;
                if (b >= tbin) cnt += __ldcg(&D.hist[b]);
            }
            s_cnt[tid] = cnt;
            __syncthreads();
            if (tid == 0) {
                unsigned K = (unsigned)D.K, cum = 0, bin = tbin;
                for (int i = 0; i < 256; ++i) {
                    if (cum + s_cnt[i] >= K) {
                        for (int j = 0; j < 16; ++j) {
                            unsigned b = STAB_HBINS - 1 - 16 * i - j;
                            if (b < tbin) break;
                            cum += __ldcg(&D.hist[b]);
                            if (cum >= K) { bin = b; break; }
                        }
                        break;
                    }
                    cum += s_cnt[i];
                }
                st->bin_lo = bin > tbin ? bin : tbin;
                st->thr_bits = thr_bits;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_filter(const StreamDev *__restrict__ S, WorkList wl)
{
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
    static int occ = 0;
    if (!occ && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_response, 256, 0) != cudaSuccess || occ < 1))
        occ = 1;
    return occ;
}

static void select_attr()
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, STAB_SEL_SMEM * 8);
        attr = true;
    }
}

void warm_detect()
{
    occ_response();
    select_attr();
}

void launch_response(const Launch &L, const StreamDev *S, WorkList wl, DetIO io)
{
    k_response<<<grid_for(L, wl.total, occ_response()), 256, 0, L.stream>>>(S, wl, io);
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

// k_warp.cu -- compensating bilinear warp (Sec. 5.1, final step): every output
// pixel p takes the source at q = Minv p, taps outside the image read 0, and
// the value is rounded half up.  The output byte is a quantised decision, so
// the FP32 operation sequence is fixed (fma for the mapping, three lerps,
// floor(v + 0.5)) and reproducible bit for bit.
//
// Persistent grid-stride loop over 64 x 16 output tiles of every stream; each
// thread writes 4 consecutive pixels with one 4-byte (gray) or three 4-byte
// (RGB) stores.  Source taps go through the read-only cache: for the small
// rotations of stabilisation neighbouring threads touch neighbouring bytes.
#include "kernels.cuh"

namespace {

template <int C>
__device__ __forceinline__ void warp_px(const uint8_t *__restrict__ src, int sp, int w, int h, const float M[6],
                                        int x, int y, uint8_t o[C])
{
    const float xf = (float)x, yf = (float)y;
    const float qx = __fmaf_rn(M[0], xf, __fmaf_rn(M[1], yf, M[2]));
    const float qy = __fmaf_rn(M[3], xf, __fmaf_rn(M[4], yf, M[5]));
    if (!(qx > -1.0f && qx < (float)w && qy > -1.0f && qy < (float)h)) {
#pragma unroll
        for (int c = 0; c < C; ++c) o[c] = 0;
        return;
    }
    const float fx = floorf(qx), fy = floorf(qy);
    const float ax = __fsub_rn(qx, fx), ay = __fsub_rn(qy, fy);
    const int x0 = (int)fx, y0 = (int)fy;
    const bool vx0 = x0 >= 0, vx1 = x0 + 1 < w, vy0 = y0 >= 0, vy1 = y0 + 1 < h;
    const uint8_t *r0 = src + (size_t)y0 * sp + (size_t)x0 * C;
    const uint8_t *r1 = r0 + sp;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float p00 = (vx0 && vy0) ? (float)__ldg(r0 + c) : 0.f;
        const float p01 = (vx1 && vy0) ? (float)__ldg(r0 + C + c) : 0.f;
        const float p10 = (vx0 && vy1) ? (float)__ldg(r1 + c) : 0.f;
        const float p11 = (vx1 && vy1) ? (float)__ldg(r1 + C + c) : 0.f;
        const float top = __fmaf_rn(ax, __fsub_rn(p01, p00), p00);
        const float bot = __fmaf_rn(ax, __fsub_rn(p11, p10), p10);
        const float v = __fmaf_rn(ay, __fsub_rn(bot, top), top);
        const float r = floorf(__fadd_rn(v, 0.5f));
        o[c] = (uint8_t)(r < 0.f ? 0 : (r > 255.f ? 255 : (int)r));
    }
}

template <int C>
__device__ __forceinline__ void warp_tile(const uint8_t *__restrict__ src, int sp, uint8_t *__restrict__ dst,
                                          int dp, int w, int h, const float M[6], int x0, int y0)
{
    const int row = threadIdx.x >> 4, x = x0 + (threadIdx.x & 15) * 4, y = y0 + row;
    if (y >= h || x >= w) return;
    uint8_t o[4 * C];
#pragma unroll
    for (int k = 0; k < 4; ++k) warp_px<C>(src, sp, w, h, M, x + k, y, o + C * k);
    uint8_t *d = dst + (size_t)y * dp + (size_t)x * C;
    const bool aligned = x + 4 <= w && ((reinterpret_cast<uintptr_t>(d) & 3) == 0);
    if (aligned) {
#pragma unroll
        for (int k = 0; k < C; ++k)
            reinterpret_cast<unsigned *>(d)[k] = (unsigned)o[4 * k] | ((unsigned)o[4 * k + 1] << 8) |
                                                 ((unsigned)o[4 * k + 2] << 16) | ((unsigned)o[4 * k + 3] << 24);
    } else {
        const int n = min(4, w - x) * C;
        for (int k = 0; k < n; ++k) d[k] = o[k];
    }
}

__global__ void __launch_bounds__(256) k_warp(const StreamDev *__restrict__ S, WorkList wl, WarpIO io)
{
    for (int item = blockIdx.x; item < wl.total; item += gridDim.x) {
        const int s = wl_stream(wl, item);
        const StreamDev &D = S[s];
        const int local = item - __ldg(&wl.prefix[s]);
        const uint8_t *src;
        uint8_t *dst;
        int sp, dp, C;
        const float *Mp;
        if (io.src) {
            src = io.src; sp = io.sp; dst = io.dst; dp = io.dp; C = io.C; Mp = io.Minv;
        } else {
            const int u = D.st->out_frame;
            if (u < 0) continue;
            src = D.ring + (long long)(u % D.ring_len) * D.slot_bytes;
            sp = D.in_pitch; dst = D.out; dp = D.out_pitch; C = D.C; Mp = D.Minv;
        }
        float M[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) M[k] = Mp[k];
        const int tx = (D.w + STAB_TW - 1) / STAB_TW;
        const int x0 = (local % tx) * STAB_TW, y0 = (local / tx) * STAB_TH;
        if (C == 3) warp_tile<3>(src, sp, dst, dp, D.w, D.h, M, x0, y0);
        else warp_tile<1>(src, sp, dst, dp, D.w, D.h, M, x0, y0);
    }
}

}  // namespace

static int occ_warp()
{
    static int occ = 0;
    if (!occ && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_warp, 256, 0) != cudaSuccess || occ < 1))
        occ = 1;
    return occ;
}

void warm_warp() { occ_warp(); }

void launch_warp(const Launch &L, const StreamDev *S, WorkList wl, WarpIO io)
{
    k_warp<<<grid_for(L, wl.total, occ_warp()), 256, 0, L.stream>>>(S, wl, io);
}

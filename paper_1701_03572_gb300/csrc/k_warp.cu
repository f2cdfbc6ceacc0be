// k_warp.cu -- compensating bilinear warp (Sec. 5.1, final step): every output
// pixel p takes the source at q = Minv p, taps outside the image read 0, and
// the value is rounded half up.  The output byte is a quantised decision, so
// the FP32 operation sequence is fixed (fma for the mapping, three lerps,
// floor(v + 0.5)) and reproducible bit for bit.
//
// Persistent grid-stride loop over 64 x 16 output tiles of every stream; each
// thread writes 4 consecutive pixels with one 4-byte (gray) or three 4-byte
// (RGB) stores.  The tile's source box is staged in shared memory with aligned
// 16-byte loads and the taps are gathered from there; tiles whose box is too
// large to stage (strong rotation or zoom) gather through the read-only cache.
#include "kernels.cuh"

namespace {

// Staging capacity for an interior tile's source box: 40 rows of 400 bytes
// (133 RGB / 400 gray pixels), enough for rotations of ~25 degrees at scale ~1.
constexpr int WS_ROWS = 40, WS_BYTES = 400;

// Bilinear value of channel taps p00 p01 (row y0), p10 p11 (row y0 + 1),
// rounded half up; v stays in [0, 255] (convex combination of bytes with
// monotone rounding), so floor(v + 0.5) needs no clamp.
__device__ __forceinline__ uint8_t lerp_round(float ax, float ay, float p00, float p01, float p10, float p11)
{
    const float top = __fmaf_rn(ax, __fsub_rn(p01, p00), p00);
    const float bot = __fmaf_rn(ax, __fsub_rn(p11, p10), p10);
    const float v = __fmaf_rn(ay, __fsub_rn(bot, top), top);
    return (uint8_t)__float2int_rd(__fadd_rn(v, 0.5f));
}

// Store the 4 C bytes o (n of them inside the row) with 32-bit stores when
// whole and aligned; loops are unrolled so o stays in registers.
template <int C>
__device__ __forceinline__ void store4(uint8_t *d, const uint8_t (&o)[4 * C], int n)
{
    if (n == 4 * C && (reinterpret_cast<uintptr_t>(d) & 3) == 0) {
#pragma unroll
        for (int k = 0; k < C; ++k)
            reinterpret_cast<unsigned *>(d)[k] = (unsigned)o[4 * k] | ((unsigned)o[4 * k + 1] << 8) |
                                                 ((unsigned)o[4 * k + 2] << 16) | ((unsigned)o[4 * k + 3] << 24);
    } else {
#pragma unroll
        for (int k = 0; k < 4 * C; ++k)
            if (k < n) d[k] = o[k];
    }
}

// General path: taps read through the read-only cache, each checked against
// the image (outside reads 0).
template <int C>
__device__ __forceinline__ void warp_tile_direct(const uint8_t *__restrict__ src, int sp, uint8_t *__restrict__ dst,
                                                 int dp, int w, int h, const float M[6], int x0, int y0)
{
    const int row = threadIdx.x >> 4, x = x0 + (threadIdx.x & 15) * 4, y = y0 + row;
    if (y >= h || x >= w) return;
    const float yf = (float)y;
    const float qx0 = __fmaf_rn(M[1], yf, M[2]), qy0 = __fmaf_rn(M[4], yf, M[5]);
    uint8_t o[4 * C];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float xf = (float)(x + k);
        const float qx = __fmaf_rn(M[0], xf, qx0), qy = __fmaf_rn(M[3], xf, qy0);
        if (!(qx > -1.0f && qx < (float)w && qy > -1.0f && qy < (float)h)) {
#pragma unroll
            for (int c = 0; c < C; ++c) o[C * k + c] = 0;
            continue;
        }
        const float fx = floorf(qx), fy = floorf(qy);
        const float ax = __fsub_rn(qx, fx), ay = __fsub_rn(qy, fy);
        const int xa = (int)fx, ya = (int)fy;
        const bool v00 = xa >= 0 && ya >= 0, v01 = xa + 1 < w && ya >= 0;
        const bool v10 = xa >= 0 && ya + 1 < h, v11 = xa + 1 < w && ya + 1 < h;
        const uint8_t *r0 = src + (size_t)ya * sp + (size_t)xa * C;
        const uint8_t *r1 = r0 + sp;
#pragma unroll
        for (int c = 0; c < C; ++c)
            o[C * k + c] = lerp_round(ax, ay, v00 ? (float)__ldg(r0 + c) : 0.f, v01 ? (float)__ldg(r0 + C + c) : 0.f,
                                      v10 ? (float)__ldg(r1 + c) : 0.f, v11 ? (float)__ldg(r1 + C + c) : 0.f);
    }
    store4<C>(dst + (size_t)y * dp + (size_t)x * C, o, min(4, w - x) * C);
}

// Interior path: every tap of the tile lies in the staged box (which lies in
// the image), so taps are plain shared-memory byte loads.
template <int C>
__device__ __forceinline__ void warp_tile_staged(const uint8_t *__restrict__ sb, int bx0, int by0, int b0,
                                                 uint8_t *__restrict__ dst, int dp, int w, int h, const float M[6],
                                                 int x0, int y0)
{
    const int row = threadIdx.x >> 4, x = x0 + (threadIdx.x & 15) * 4, y = y0 + row;
    if (y >= h || x >= w) return;
    const float yf = (float)y;
    const float qx0 = __fmaf_rn(M[1], yf, M[2]), qy0 = __fmaf_rn(M[4], yf, M[5]);
    uint8_t o[4 * C];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float xf = (float)(x + k);
        const float qx = __fmaf_rn(M[0], xf, qx0), qy = __fmaf_rn(M[3], xf, qy0);
        const float fx = floorf(qx), fy = floorf(qy);
        const float ax = __fsub_rn(qx, fx), ay = __fsub_rn(qy, fy);
        const uint8_t *r0 = sb + ((int)fy - by0) * WS_BYTES + ((int)fx * C - b0);
        const uint8_t *r1 = r0 + WS_BYTES;
#pragma unroll
        for (int c = 0; c < C; ++c)
            o[C * k + c] = lerp_round(ax, ay, (float)r0[c], (float)r0[C + c], (float)r1[c], (float)r1[C + c]);
    }
    store4<C>(dst + (size_t)y * dp + (size_t)x * C, o, min(4, w - x) * C);
}

// Box of the taps of an output tile: the mapped tile corners (the map is
// affine) widened by one pixel for the right / lower tap and one more for
// rounding.
__device__ __forceinline__ void tile_box(const float M[6], int x0, int y0, int w, int h, int &bx0, int &by0,
                                         int &bx1, int &by1)
{
    const float xa = (float)x0, xb = (float)min(x0 + STAB_TW - 1, w - 1);
    const float ya = (float)y0, yb = (float)min(y0 + STAB_TH - 1, h - 1);
    float qx[4], qy[4];
    qx[0] = M[0] * xa + M[1] * ya + M[2]; qy[0] = M[3] * xa + M[4] * ya + M[5];
    qx[1] = M[0] * xb + M[1] * ya + M[2]; qy[1] = M[3] * xb + M[4] * ya + M[5];
    qx[2] = M[0] * xa + M[1] * yb + M[2]; qy[2] = M[3] * xa + M[4] * yb + M[5];
    qx[3] = M[0] * xb + M[1] * yb + M[2]; qy[3] = M[3] * xb + M[4] * yb + M[5];
    float mnx = fminf(fminf(qx[0], qx[1]), fminf(qx[2], qx[3])), mxx = fmaxf(fmaxf(qx[0], qx[1]), fmaxf(qx[2], qx[3]));
    float mny = fminf(fminf(qy[0], qy[1]), fminf(qy[2], qy[3])), mxy = fmaxf(fmaxf(qy[0], qy[1]), fmaxf(qy[2], qy[3]));
    mnx = fminf(fmaxf(mnx, -8.f), (float)w + 8.f); mxx = fminf(fmaxf(mxx, -8.f), (float)w + 8.f);
    mny = fminf(fmaxf(mny, -8.f), (float)h + 8.f); mxy = fminf(fmaxf(mxy, -8.f), (float)h + 8.f);
    bx0 = (int)floorf(mnx) - 1;
    by0 = (int)floorf(mny) - 1;
    bx1 = (int)floorf(mxx) + 2;
    by1 = (int)floorf(mxy) + 2;
}

__global__ void __launch_bounds__(256) k_warp(const StreamDev *__restrict__ S, WorkList wl, WarpIO io)
{
    __shared__ __align__(16) uint8_t sbox[WS_ROWS * WS_BYTES];
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
        const int w = D.w, h = D.h;
        const int tx = (w + STAB_TW - 1) / STAB_TW;
        const int x0 = (local % tx) * STAB_TW, y0 = (local / tx) * STAB_TH;
        int bx0, by0, bx1, by1;
        tile_box(M, x0, y0, w, h, bx0, by0, bx1, by1);
        const int b0 = (bx0 * C) & ~15, nvec = ((bx1 + 1) * C - b0 + 15) >> 4, rows = by1 - by0 + 1;
        const bool interior = bx0 >= 0 && by0 >= 0 && bx1 <= w - 1 && by1 <= h - 1 && rows <= WS_ROWS &&
                              nvec * 16 <= WS_BYTES && b0 + nvec * 16 <= sp &&
                              ((reinterpret_cast<uintptr_t>(src) | (uintptr_t)sp) & 15) == 0;
        if (interior) {
            for (int e = threadIdx.x; e < rows * nvec; e += blockDim.x) {
                const int r = e / nvec, v = e - r * nvec;
                *reinterpret_cast<uint4 *>(sbox + r * WS_BYTES + 16 * v) =
                    __ldg(reinterpret_cast<const uint4 *>(src + (size_t)(by0 + r) * sp + b0) + v);
            }
            __syncthreads();
            if (C == 3) warp_tile_staged<3>(sbox, bx0, by0, b0, dst, dp, w, h, M, x0, y0);
            else warp_tile_staged<1>(sbox, bx0, by0, b0, dst, dp, w, h, M, x0, y0);
            __syncthreads();
        } else {
            if (C == 3) warp_tile_direct<3>(src, sp, dst, dp, w, h, M, x0, y0);
            else warp_tile_direct<1>(src, sp, dst, dp, w, h, M, x0, y0);
        }
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

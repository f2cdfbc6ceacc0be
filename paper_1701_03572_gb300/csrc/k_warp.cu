// k_warp.cu -- compensating bilinear warp (Sec. 5.1, final step): every output
// pixel p takes the source at q = Minv p, taps outside the image read 0, and
// the value is rounded half up.  The output byte is a quantised decision, so
// the FP32 operation sequence is fixed (fma for the mapping, three lerps,
// floor(v + 0.5)) and reproducible bit for bit.
//
// Persistent grid-stride loop over 64 x 32 output tiles of every stream; each
// thread writes 4 consecutive pixels of two rows with 4-byte stores.  The
// source box of a tile is copied into shared memory with 16-byte cp.async
// (bytes outside the image zero-filled by the copy itself), one tile ahead of
// the tile being computed, so the next box streams in while this one is
// resampled.  Tiles whose box is too large to stage (strong rotation or zoom)
// gather through the read-only cache instead.
//
// No float/int conversion instruction is on the per-pixel path (they issue at
// a quarter of the FP32 rate): a byte b becomes the float 2^23 + b by placing
// it under the exponent pattern 0x4B000000, floor(q) for |q| < 2^22 is
// (q + 1.5 * 2^23 rounded down) - 1.5 * 2^23, and the final floor(v + 0.5) is
// read from the low byte of (v + 0.5) + 2^23 rounded down.  Each is exact, so
// the results equal the plain floorf / conversion forms bit for bit.
#include "kernels.cuh"

namespace {

// Staging capacity: 48 rows of 320 bytes (106 RGB / 320 gray pixels): a 64 x 32
// tile rotated by up to ~11 degrees at scale ~1.  320-byte rows are 80 words,
// 16 banks apart, so the two output rows of a warp read disjoint bank halves.
constexpr int WS_ROWS = 48, WS_BYTES = 320, WS_BUF = WS_ROWS * WS_BYTES + 16;
constexpr float kTwo23 = 8388608.0f, kFloorMagic = 12582912.0f;   // 2^23, 1.5 * 2^23
constexpr int kFloorBits = 0x4B400000;                             // bit pattern of 1.5 * 2^23

struct WJob {
    const uint8_t *src;
    uint8_t *dst;
    int sp, dp, w, h, C, x0, y0;
    int by0, b0, rows, nvec;
    int mode;      // 0 nothing to write, 1 staged, 2 direct gather
    bool edge;     // the box leaves the image: per-pixel range test
    float M[6];
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Exact floor for |q| < 2^22: value and integer.
__device__ __forceinline__ float floor_exact(float q, int &qi)
{
    const float r = __fadd_rd(q, kFloorMagic);
    qi = __float_as_int(r) - kFloorBits;
    return __fsub_rn(r, kFloorMagic);
}

// Byte `sel` of word t as the float 2^23 + byte.
template <int SEL>
__device__ __forceinline__ float byte_biased(unsigned t)
{
    return __uint_as_float(__byte_perm(t, 0x4B000000u, 0x7540 | SEL));
}

// Bilinear value from biased taps (2^23 + byte), rounded half up; returns a
// word whose low byte is the result.  top / bottom / vertical lerps are the
// same fma sequence as the unbiased form (differences of biased taps are
// exact).
__device__ __forceinline__ unsigned lerp_biased(float ax, float ay, float b00, float b01, float b10, float b11)
{
    const float top = __fmaf_rn(ax, __fsub_rn(b01, b00), __fsub_rn(b00, kTwo23));
    const float bot = __fmaf_rn(ax, __fsub_rn(b11, b10), __fsub_rn(b10, kTwo23));
    const float v = __fmaf_rn(ay, __fsub_rn(bot, top), top);
    return __float_as_uint(__fadd_rd(__fadd_rn(v, 0.5f), kTwo23));
}

// Plain form of the same rounding, for the gather path (v in [0, 255]).
__device__ __forceinline__ uint8_t lerp_round(float ax, float ay, float p00, float p01, float p10, float p11)
{
    const float top = __fmaf_rn(ax, __fsub_rn(p01, p00), p00);
    const float bot = __fmaf_rn(ax, __fsub_rn(p11, p10), p10);
    const float v = __fmaf_rn(ay, __fsub_rn(bot, top), top);
    return (uint8_t)__float2int_rd(__fadd_rn(v, 0.5f));
}

// Pack the low bytes of a, b, c, d into one word.
__device__ __forceinline__ unsigned pack4(unsigned a, unsigned b, unsigned c, unsigned d)
{
    return __byte_perm(__byte_perm(a, b, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
}

// Store 4 pixels of C bytes (words o[0 .. C-1]); n bytes lie inside the row.
template <int C>
__device__ __forceinline__ void store_px4(uint8_t *d, const unsigned (&o)[C], int n)
{
    if (n == 4 * C && (reinterpret_cast<uintptr_t>(d) & 3) == 0) {
#pragma unroll
        for (int k = 0; k < C; ++k) reinterpret_cast<unsigned *>(d)[k] = o[k];
    } else {
#pragma unroll
        for (int k = 0; k < 4 * C; ++k)
            if (k < n) d[k] = (uint8_t)(o[k >> 2] >> (8 * (k & 3)));
    }
}

// Box of the taps of an output tile: the mapped tile corners (the map is
// affine) clamped to 8 pixels around the image, widened by one pixel for
// rounding and one more for the right / lower tap.
__device__ __forceinline__ void tile_box(const float M[6], int x0, int y0, int w, int h, int &bx0, int &by0,
                                         int &bx1, int &by1)
{
    const float xa = (float)x0, xb = (float)min(x0 + STAB_TW - 1, w - 1);
    const float ya = (float)y0, yb = (float)min(y0 + STAB_WTH - 1, h - 1);
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

__device__ __forceinline__ void make_job(const StreamDev *__restrict__ S, const WorkList &wl, const WarpIO &io,
                                         int item, WJob &j)
{
    const int s = wl_stream(wl, item);
    const StreamDev &D = S[s];
    const int local = item - __ldg(&wl.prefix[s]);
    const float *Mp;
    j.mode = 0;
    if (io.src) {
        j.src = io.src; j.sp = io.sp; j.dst = io.dst; j.dp = io.dp; j.C = io.C; Mp = io.Minv;
    } else {
        const int u = D.st->out_frame;
        if (u < 0) return;
        j.src = D.ring + (long long)(u % D.ring_len) * D.slot_bytes;
        j.sp = D.in_pitch; j.dst = D.out; j.dp = D.out_pitch; j.C = D.C; Mp = D.Minv;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) j.M[k] = Mp[k];
    j.w = D.w; j.h = D.h;
    const int tx = (j.w + STAB_TW - 1) / STAB_TW;
    j.x0 = (local % tx) * STAB_TW; j.y0 = (local / tx) * STAB_WTH;
    int bx0, by0, bx1, by1;
    tile_box(j.M, j.x0, j.y0, j.w, j.h, bx0, by0, bx1, by1);
    j.by0 = by0;
    j.b0 = (bx0 * j.C) & ~15;                                  // floor to 16 bytes (bx0 may be negative)
    j.nvec = ((bx1 + 1) * j.C - j.b0 + 15) >> 4;
    j.rows = by1 - by0 + 1;
    j.edge = !(bx0 >= 0 && by0 >= 0 && bx1 <= j.w - 1 && by1 <= j.h - 1);
    const bool fits = j.rows <= WS_ROWS && j.nvec * 16 <= WS_BYTES &&
                      ((reinterpret_cast<uintptr_t>(j.src) | (uintptr_t)j.sp) & 15) == 0;
    j.mode = fits ? 1 : 2;
}

// Copy the job's box into sb: 16-byte chunk (r, v) holds row by0 + r, bytes
// b0 + 16 v .. + 15; bytes outside the image come out 0 (src-size operand).
__device__ __forceinline__ void stage(const WJob &j, uint8_t *sb)
{
    const int n = j.rows * j.nvec, rowbytes = j.w * j.C;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int r = e / j.nvec, v = e - r * j.nvec;
        const int gy = j.by0 + r, gx = j.b0 + 16 * v;
        int valid = 0;
        if (gy >= 0 && gy < j.h && gx >= 0) valid = min(16, max(0, rowbytes - gx));
        const uint8_t *g = valid ? j.src + (size_t)gy * j.sp + gx : j.src;
        cp_async16(sb + r * WS_BYTES + 16 * v, g, valid);
    }
}

// Resample a staged tile: thread (ty, tx) writes pixels x0 + 4 tx .. + 3 of
// rows y0 + ty and y0 + ty + 16.
template <int C, bool EDGE>
__device__ __forceinline__ void warp_staged(const uint8_t *__restrict__ sb, const WJob &j)
{
    const int x = j.x0 + (threadIdx.x & 15) * 4;
    if (x >= j.w) return;
    const float xf0 = (float)x, fw = (float)j.w, fh = (float)j.h;
    const int base = -j.by0 * WS_BYTES - j.b0;
#pragma unroll 1
    for (int rr = 0; rr < 2; ++rr) {
        const int y = j.y0 + (threadIdx.x >> 4) + 16 * rr;
        if (y >= j.h) break;
        const float yf = (float)y;
        const float qx0 = __fmaf_rn(j.M[1], yf, j.M[2]), qy0 = __fmaf_rn(j.M[4], yf, j.M[5]);
        unsigned res[4 * C];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float xf = __fadd_rn(xf0, (float)k);
            const float qx = __fmaf_rn(j.M[0], xf, qx0), qy = __fmaf_rn(j.M[3], xf, qy0);
            if (EDGE && !(qx > -1.0f && qx < fw && qy > -1.0f && qy < fh)) {
#pragma unroll
                for (int c = 0; c < C; ++c) res[C * k + c] = 0u;
                continue;
            }
            int xi, yi;
            const float fx = floor_exact(qx, xi), fy = floor_exact(qy, yi);
            const float ax = __fsub_rn(qx, fx), ay = __fsub_rn(qy, fy);
            const int o = base + yi * WS_BYTES + xi * C;   // byte offset of tap (xi, yi) in sb
            if (C == 3) {
                // taps (xi, xi + 1) of a row: 6 bytes at o, inside words o/4 .. o/4 + 2
                const unsigned *w0 = reinterpret_cast<const unsigned *>(sb + (o & ~3));
                const unsigned *w1 = w0 + WS_BYTES / 4;
                const unsigned sel = 0x3210u + (unsigned)(o & 3) * 0x1111u;
                const unsigned a0 = __byte_perm(w0[0], w0[1], sel), a1 = __byte_perm(w0[1], w0[2], sel);
                const unsigned c0 = __byte_perm(w1[0], w1[1], sel), c1 = __byte_perm(w1[1], w1[2], sel);
                res[3 * k + 0] = lerp_biased(ax, ay, byte_biased<0>(a0), byte_biased<3>(a0), byte_biased<0>(c0),
                                             byte_biased<3>(c0));
                res[3 * k + 1] = lerp_biased(ax, ay, byte_biased<1>(a0), byte_biased<0>(a1), byte_biased<1>(c0),
                                             byte_biased<0>(c1));
                res[3 * k + 2] = lerp_biased(ax, ay, byte_biased<2>(a0), byte_biased<1>(a1), byte_biased<2>(c0),
                                             byte_biased<1>(c1));
            } else {
                const uint8_t *r0 = sb + o, *r1 = r0 + WS_BYTES;
                res[k] = lerp_biased(ax, ay, __uint_as_float(0x4B000000u | r0[0]), __uint_as_float(0x4B000000u | r0[1]),
                                     __uint_as_float(0x4B000000u | r1[0]), __uint_as_float(0x4B000000u | r1[1]));
            }
        }
        unsigned o[C];
#pragma unroll
        for (int k = 0; k < C; ++k) o[k] = pack4(res[4 * k], res[4 * k + 1], res[4 * k + 2], res[4 * k + 3]);
        store_px4<C>(j.dst + (size_t)y * j.dp + (size_t)x * C, o, min(4, j.w - x) * C);
    }
}

// Gather path: taps read through the read-only cache, each checked against
// the image (outside reads 0).
template <int C>
__device__ __forceinline__ void warp_direct(const WJob &j)
{
    const int x = j.x0 + (threadIdx.x & 15) * 4;
    if (x >= j.w) return;
    const int w = j.w, h = j.h;
#pragma unroll 1
    for (int rr = 0; rr < 2; ++rr) {
        const int y = j.y0 + (threadIdx.x >> 4) + 16 * rr;
        if (y >= h) break;
        const float yf = (float)y;
        const float qx0 = __fmaf_rn(j.M[1], yf, j.M[2]), qy0 = __fmaf_rn(j.M[4], yf, j.M[5]);
        uint8_t ob[4 * C];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float xf = (float)(x + k);
            const float qx = __fmaf_rn(j.M[0], xf, qx0), qy = __fmaf_rn(j.M[3], xf, qy0);
            if (!(qx > -1.0f && qx < (float)w && qy > -1.0f && qy < (float)h)) {
#pragma unroll
                for (int c = 0; c < C; ++c) ob[C * k + c] = 0;
                continue;
            }
            const float fx = floorf(qx), fy = floorf(qy);
            const float ax = __fsub_rn(qx, fx), ay = __fsub_rn(qy, fy);
            const int xa = (int)fx, ya = (int)fy;
            const bool v00 = xa >= 0 && ya >= 0, v01 = xa + 1 < w && ya >= 0;
            const bool v10 = xa >= 0 && ya + 1 < h, v11 = xa + 1 < w && ya + 1 < h;
            const uint8_t *r0 = j.src + (long long)ya * j.sp + (long long)xa * C;
            const uint8_t *r1 = r0 + j.sp;
#pragma unroll
            for (int c = 0; c < C; ++c)
                ob[C * k + c] = lerp_round(ax, ay, v00 ? (float)__ldg(r0 + c) : 0.f, v01 ? (float)__ldg(r0 + C + c) : 0.f,
                                           v10 ? (float)__ldg(r1 + c) : 0.f, v11 ? (float)__ldg(r1 + C + c) : 0.f);
        }
        unsigned o[C];
#pragma unroll
        for (int k = 0; k < C; ++k) o[k] = pack4(ob[4 * k], ob[4 * k + 1], ob[4 * k + 2], ob[4 * k + 3]);
        store_px4<C>(j.dst + (size_t)y * j.dp + (size_t)x * C, o, min(4, w - x) * C);
    }
}

__global__ void __launch_bounds__(256) k_warp(const StreamDev *__restrict__ S, WorkList wl, WarpIO io)
{
    __shared__ __align__(16) uint8_t sbox[2][WS_BUF];
    __shared__ WJob sjob[2];   // every thread derives the same job; thread 0 publishes it for the compute
    int item = blockIdx.x;
    {
        WJob j;
        j.mode = 0;
        if (item < wl.total) {
            make_job(S, wl, io, item, j);
            if (j.mode == 1) stage(j, sbox[0]);
        }
        if (threadIdx.x == 0) sjob[0] = j;
    }
    cp_async_commit();
    for (int it = 0; item < wl.total; item += gridDim.x, ++it) {
        // the next tile's box streams into the other buffer while this one is resampled
        const int nitem = item + gridDim.x;
        {
            WJob j;
            j.mode = 0;
            if (nitem < wl.total) {
                make_job(S, wl, io, nitem, j);
                if (j.mode == 1) stage(j, sbox[(it + 1) & 1]);
            }
            if (threadIdx.x == 0) sjob[(it + 1) & 1] = j;
        }
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const WJob &cur = sjob[it & 1];
        const uint8_t *sb = sbox[it & 1];
        const int mode = cur.mode, C = cur.C;
        if (mode == 1) {
            if (C == 3) {
                if (cur.edge) warp_staged<3, true>(sb, cur);
                else warp_staged<3, false>(sb, cur);
            } else {
                if (cur.edge) warp_staged<1, true>(sb, cur);
                else warp_staged<1, false>(sb, cur);
            }
        } else if (mode == 2) {
            if (C == 3) warp_direct<3>(cur);
            else warp_direct<1>(cur);
        }
        __syncthreads();   // this buffer and job slot are refilled by the prefetch two tiles on
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

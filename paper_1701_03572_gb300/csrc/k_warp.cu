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
// the results equal the plain floorf / conversion forms bit for bit.  The FP32
// arithmetic runs on pixel pairs with the packed f32x2 forms of add / sub / fma
// (each lane the same IEEE operation, so again the same bits).  One warp
// derives each tile's job (stream, map, source box) two tiles ahead and
// publishes it in shared memory.
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
    int vq, vr, vinv;   // 256 / nvec, 256 % nvec, ceil(2^16 / nvec): the staging loop's stride
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

// Bilinear values of two pixels from biased taps (2^23 + byte), rounded half
// up; the low byte of each lane's bits is the result.  The lerps are the fma
// sequence of the plain form (differences of biased taps are exact, and the
// unbiased corner is tap - 2^23).
__device__ __forceinline__ fx2 lerp2(fx2 ax, fx2 ay, fx2 b00, fx2 b01, fx2 b10, fx2 b11)
{
    const fx2 t23 = pk(kTwo23, kTwo23), half = pk(0.5f, 0.5f);
    const fx2 top = fma2(ax, sub2(b01, b00), sub2(b00, t23));
    const fx2 bot = fma2(ax, sub2(b11, b10), sub2(b10, t23));
    const fx2 v = fma2(ay, sub2(bot, top), top);
    return add2_rd(add2(v, half), t23);
}

// Byte `sel` of word t as the float 2^23 + byte.
template <int SEL>
__device__ __forceinline__ float byte_biased(unsigned t)
{
    return __uint_as_float(__byte_perm(t, 0x4B000000u, 0x7540 | SEL));
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

// Per-stream facts a tile's job needs, gathered once per block into shared
// memory (batches of up to 64 streams), so that deriving a job reads shared
// memory only.
constexpr int WT_MAXS = 64;
struct WStream {
    const uint8_t *src;
    uint8_t *dst;
    int sp, dp, w, h, C, first, valid;
    float M[6];
};

__device__ __forceinline__ WStream stream_facts(const StreamDev *__restrict__ S, const WarpIO &io, const WorkList &wl,
                                                int s)
{
    const StreamDev &D = S[s];
    WStream f;
    f.w = D.w; f.h = D.h; f.first = __ldg(&wl.prefix[s]); f.valid = 1;
    const float *Mp;
    if (io.src) {
        f.src = io.src; f.sp = io.sp; f.dst = io.dst; f.dp = io.dp; f.C = io.C; Mp = io.Minv;
    } else {
        // the frame and map the previous step's fit produced (this step's fit is
        // writing the other slot)
        const long long t = D.st->t;
        const int slot = (int)((t - 1) & 1);
        const int u = t >= 1 ? D.st->out_frame[slot] : -1;
        f.valid = u >= 0;
        f.src = D.ring + (long long)(max(u, 0) % D.ring_len) * D.slot_bytes;
        // two output buffers by step parity: the host copy of one overlaps the next step
        f.sp = D.in_pitch; f.dst = D.out + (long long)(D.st->t & 1) * D.slot_bytes; f.dp = D.out_pitch; f.C = D.C;
        Mp = D.Minv + 8 * slot;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) f.M[k] = Mp[k];
    return f;
}

__device__ __forceinline__ void make_job(const StreamDev *__restrict__ S, const WorkList &wl, const WarpIO &io,
                                         const WStream *tab, int item, WJob &j)
{
    j.mode = 0;
    WStream f;
    if (tab) {   // stream of the item by binary search of the first items in shared memory
        int lo = 0, hi = wl.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab[mid].first <= item) lo = mid;
            else hi = mid - 1;
        }
        f = tab[lo];
    } else {
        f = stream_facts(S, io, wl, wl_stream(wl, item));
    }
    if (!f.valid) return;
    const int local = item - f.first;
    j.src = f.src; j.sp = f.sp; j.dst = f.dst; j.dp = f.dp; j.C = f.C; j.w = f.w; j.h = f.h;
#pragma unroll
    for (int k = 0; k < 6; ++k) j.M[k] = f.M[k];
    const int tx = (j.w + STAB_TW - 1) / STAB_TW;
    j.x0 = (local % tx) * STAB_TW; j.y0 = (local / tx) * STAB_WTH;
    int bx0, by0, bx1, by1;
    tile_box(j.M, j.x0, j.y0, j.w, j.h, bx0, by0, bx1, by1);
    j.by0 = by0;
    j.b0 = (bx0 * j.C) & ~15;                                  // floor to 16 bytes (bx0 may be negative)
    j.nvec = ((bx1 + 1) * j.C - j.b0 + 15) >> 4;
    j.rows = by1 - by0 + 1;
    j.vq = 256 / j.nvec; j.vr = 256 - j.vq * j.nvec; j.vinv = (65536 + j.nvec - 1) / j.nvec;
    j.edge = !(bx0 >= 0 && by0 >= 0 && bx1 <= j.w - 1 && by1 <= j.h - 1);
    const bool fits = j.rows <= WS_ROWS && j.nvec * 16 <= WS_BYTES &&
                      ((reinterpret_cast<uintptr_t>(j.src) | (uintptr_t)j.sp) & 15) == 0;
    j.mode = fits ? 1 : 2;
}

// Copy the job's box into sb: 16-byte chunk (r, v) holds row by0 + r, bytes
// b0 + 16 v .. + 15; bytes outside the image come out 0 (src-size operand).
// (256 threads; chunk e = threadIdx.x + 256 k, row = e / nvec stepped by the
// job's precomputed quotient and remainder of 256 / nvec; tid / nvec by the
// reciprocal, exact for tid < 256 and nvec < 256.)
__device__ __forceinline__ void stage(const WJob &j, uint8_t *sb)
{
    const int nv = j.nvec, n = j.rows * nv, rowbytes = j.w * j.C, h = j.h, by0 = j.by0, b0 = j.b0, sp = j.sp;
    const int vq = j.vq, vr = j.vr;
    const uint8_t *src = j.src;
    int r = (int)((threadIdx.x * (unsigned)j.vinv) >> 16), v = threadIdx.x - r * nv;
    for (int e = threadIdx.x; e < n; e += 256) {
        const int gy = by0 + r, gx = b0 + 16 * v;
        int valid = 0;
        if (gy >= 0 && gy < h && gx >= 0) valid = min(16, max(0, rowbytes - gx));
        const uint8_t *g = valid ? src + (size_t)gy * sp + gx : src;
        cp_async16(sb + r * WS_BYTES + 16 * v, g, valid);
        v += vr; r += vq;
        if (v >= nv) { v -= nv; ++r; }
    }
}

// Resample a staged tile: thread (ty, tx) writes pixels x0 + 4 tx .. + 3 of
// rows y0 + ty and y0 + ty + 16, as the pixel pairs (0, 1) and (2, 3).
template <int C, bool EDGE>
__device__ __forceinline__ void warp_staged(const uint8_t *__restrict__ sb, const WJob &j)
{
    const int x = j.x0 + (threadIdx.x & 15) * 4, w = j.w, h = j.h;
    if (x >= w) return;
    const float xf0 = (float)x, fw = (float)w, fh = (float)h;
    const int base = -j.by0 * WS_BYTES - j.b0;
    const float m0 = j.M[0], m1 = j.M[1], m2 = j.M[2], m3 = j.M[3], m4 = j.M[4], m5 = j.M[5];
    const fx2 M0 = pk(m0, m0), M3 = pk(m3, m3), MAG = pk(kFloorMagic, kFloorMagic);
    const fx2 X01 = pk(xf0, __fadd_rn(xf0, 1.f)), X23 = pk(__fadd_rn(xf0, 2.f), __fadd_rn(xf0, 3.f));
    uint8_t *drow = j.dst + (size_t)x * C;
#pragma unroll 1
    for (int rr = 0; rr < 2; ++rr) {
        const int y = j.y0 + (threadIdx.x >> 4) + 16 * rr;
        if (y >= h) break;
        const float yf = (float)y;
        const float qx0 = __fmaf_rn(m1, yf, m2), qy0 = __fmaf_rn(m4, yf, m5);
        const fx2 QX0 = pk(qx0, qx0), QY0 = pk(qy0, qy0);
        unsigned res[4 * C];
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
            const fx2 qx = fma2(M0, pp ? X23 : X01, QX0), qy = fma2(M3, pp ? X23 : X01, QY0);
            const fx2 rx = add2_rd(qx, MAG), ry = add2_rd(qy, MAG);
            const fx2 ax = sub2(qx, sub2(rx, MAG)), ay = sub2(qy, sub2(ry, MAG));
            float q[2][2], rf[2][2];
            upk(qx, q[0][0], q[1][0]); upk(qy, q[0][1], q[1][1]);
            upk(rx, rf[0][0], rf[1][0]); upk(ry, rf[0][1], rf[1][1]);
            bool ok[2];
            int o[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                ok[e] = !EDGE || (q[e][0] > -1.0f && q[e][0] < fw && q[e][1] > -1.0f && q[e][1] < fh);
                const int xi = __float_as_int(rf[e][0]) - kFloorBits, yi = __float_as_int(rf[e][1]) - kFloorBits;
                o[e] = ok[e] ? base + yi * WS_BYTES + xi * C : 0;   // a pixel outside reads nothing it uses
            }
            if (C == 3) {
                // taps (xi, xi + 1) of a row: 6 bytes at o, inside words o/4 .. o/4 + 2
                unsigned a0[2], a1[2], c0[2], c1[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const unsigned *w0 = reinterpret_cast<const unsigned *>(sb + (o[e] & ~3));
                    const unsigned *w1 = w0 + WS_BYTES / 4;
                    const unsigned sel = 0x3210u + (unsigned)(o[e] & 3) * 0x1111u;
                    a0[e] = __byte_perm(w0[0], w0[1], sel); a1[e] = __byte_perm(w0[1], w0[2], sel);
                    c0[e] = __byte_perm(w1[0], w1[1], sel); c1[e] = __byte_perm(w1[1], w1[2], sel);
                }
                const fx2 r0 = lerp2(ax, ay, pk(byte_biased<0>(a0[0]), byte_biased<0>(a0[1])),
                                    pk(byte_biased<3>(a0[0]), byte_biased<3>(a0[1])),
                                    pk(byte_biased<0>(c0[0]), byte_biased<0>(c0[1])),
                                    pk(byte_biased<3>(c0[0]), byte_biased<3>(c0[1])));
                const fx2 r1 = lerp2(ax, ay, pk(byte_biased<1>(a0[0]), byte_biased<1>(a0[1])),
                                    pk(byte_biased<0>(a1[0]), byte_biased<0>(a1[1])),
                                    pk(byte_biased<1>(c0[0]), byte_biased<1>(c0[1])),
                                    pk(byte_biased<0>(c1[0]), byte_biased<0>(c1[1])));
                const fx2 r2 = lerp2(ax, ay, pk(byte_biased<2>(a0[0]), byte_biased<2>(a0[1])),
                                    pk(byte_biased<1>(a1[0]), byte_biased<1>(a1[1])),
                                    pk(byte_biased<2>(c0[0]), byte_biased<2>(c0[1])),
                                    pk(byte_biased<1>(c1[0]), byte_biased<1>(c1[1])));
                float v[3][2];
                upk(r0, v[0][0], v[0][1]); upk(r1, v[1][0], v[1][1]); upk(r2, v[2][0], v[2][1]);
#pragma unroll
                for (int e = 0; e < 2; ++e)
#pragma unroll
                    for (int c = 0; c < 3; ++c) res[3 * (2 * pp + e) + c] = ok[e] ? __float_as_uint(v[c][e]) : 0u;
            } else {
                const uint8_t *p0 = sb + o[0], *p1 = sb + o[1];
                const fx2 r0 = lerp2(ax, ay, pk(__uint_as_float(0x4B000000u | p0[0]), __uint_as_float(0x4B000000u | p1[0])),
                                    pk(__uint_as_float(0x4B000000u | p0[1]), __uint_as_float(0x4B000000u | p1[1])),
                                    pk(__uint_as_float(0x4B000000u | p0[WS_BYTES]), __uint_as_float(0x4B000000u | p1[WS_BYTES])),
                                    pk(__uint_as_float(0x4B000000u | p0[WS_BYTES + 1]),
                                       __uint_as_float(0x4B000000u | p1[WS_BYTES + 1])));
                float v0, v1;
                upk(r0, v0, v1);
                res[2 * pp] = ok[0] ? __float_as_uint(v0) : 0u;
                res[2 * pp + 1] = ok[1] ? __float_as_uint(v1) : 0u;
            }
        }
        unsigned o[C];
#pragma unroll
        for (int k = 0; k < C; ++k) o[k] = pack4(res[4 * k], res[4 * k + 1], res[4 * k + 2], res[4 * k + 3]);
        store_px4<C>(drow + (size_t)y * j.dp, o, min(4, w - x) * C);
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

__global__ void __launch_bounds__(256, 4) k_warp(const StreamDev *__restrict__ S, WorkList wl, WarpIO io)
{
    __shared__ __align__(16) uint8_t sbox[2][WS_BUF];
    __shared__ WJob sjob[3];   // jobs of tiles it, it + 1, it + 2 (slot k % 3), derived by warp 0
    __shared__ WStream stab[WT_MAXS];
    const WStream *tab = wl.n <= WT_MAXS ? stab : nullptr;
    if (tab)
        for (int s = threadIdx.x; s < wl.n; s += blockDim.x) stab[s] = stream_facts(S, io, wl, s);
    __syncthreads();
    const int G = gridDim.x;
    int item = blockIdx.x;
    if (threadIdx.x < 32) {
        for (int k = 0; k < 2; ++k) {
            WJob j;
            j.mode = 0;
            if (item + k * G < wl.total) make_job(S, wl, io, tab, item + k * G, j);
            if (threadIdx.x == 0) sjob[k] = j;
        }
    }
    __syncthreads();
    if (sjob[0].mode == 1) stage(sjob[0], sbox[0]);
    cp_async_commit();
    for (int it = 0; item < wl.total; item += G, ++it) {
        // the next tile's box streams into the other buffer while this one is resampled
        const WJob &nxt = sjob[(it + 1) % 3];
        if (nxt.mode == 1) stage(nxt, sbox[(it + 1) & 1]);
        cp_async_commit();
        if (threadIdx.x < 32) {
            WJob j;
            j.mode = 0;
            if (item + 2 * G < wl.total) make_job(S, wl, io, tab, item + 2 * G, j);
            if (threadIdx.x == 0) sjob[(it + 2) % 3] = j;
        }
        cp_async_wait1();
        __syncthreads();
        const WJob &cur = sjob[it % 3];
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
        __syncthreads();   // this buffer and job slot are refilled two tiles on
    }
}

}  // namespace

static int occ_warp()
{
    static DevCache c;
    return c.get([] {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_warp, 256, 0) != cudaSuccess || occ < 1) occ = 1;
        return occ;
    });
}

void warm_warp() { occ_warp(); }

void launch_warp(const Launch &L, const StreamDev *S, WorkList wl, WarpIO io)
{
    k_warp<<<grid_for(L, wl.total, occ_warp()), 256, 0, L.stream>>>(S, wl, io);
}

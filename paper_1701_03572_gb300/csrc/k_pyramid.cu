// k_pyramid.cu -- Gaussian pyramid (Sec. 3.2; Burt-Adelson REDUCE with the
// generating kernel [1 4 6 4 1] / 16) and the I / Ix / Iy planes the tracker
// reads (central differences, replicated border), in FP32 or FP16 storage.
//
// Both kernels are persistent grid-stride loops over a work list of vertical
// strips spanning every stream of the batch, with no shared memory and no
// barrier: a thread walks down 4 consecutive columns, keeping the rows it
// still needs in registers, and emits each row's 4 pixels with vector stores
// (one word for the u8 level, float4 / uint2 for I, 2 x float4 / uint4 for the
// gradient pair).  The integer blur is exact, so every level is bit-identical
// to the definition; FP16 holds the integers and half-integers of I and its
// central differences exactly, so both storages carry the same values.
#include "kernels.cuh"

namespace {

__device__ __forceinline__ int reflect101(int i, int n)
{
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * n - 2 - i;
    }
    return i;
}

__device__ __forceinline__ void store_I(float *p, const float v[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store_G(float2 *p, const float gx[4], const float gy[4])
{
    float4 *q = reinterpret_cast<float4 *>(p);
    q[0] = make_float4(gx[0], gy[0], gx[1], gy[1]);
    q[1] = make_float4(gx[2], gy[2], gx[3], gy[3]);
}

// Level 0: frame (gray, or RGB converted to luma) -> u8 level 0 + planes.
// Vertical strips, no shared memory and no barriers: a thread owns 4
// consecutive columns x .. x+3 of a STAB_L0_ROWS-row strip and walks down it with the
// luma of rows y-1, y, y+1 (columns x-1 .. x+4) in registers; each new row
// costs five aligned 32-bit loads of RGB (three of gray), each emitted row
// three vector stores.  Columns and rows outside the image are clamped
// (replicated border), so the planes match the clamped central differences.
constexpr int L0_STRIP = STAB_L0_ROWS;   // rows per strip
constexpr int L0_GROUPS = 128; // 4-column groups per work item (one per thread)

__device__ __forceinline__ unsigned luma4(unsigned a, unsigned b, unsigned c)
{
    // 12 bytes = 4 RGB pixels: a = r0 g0 b0 r1, b = g1 b1 r2 g2, c = b2 r3 g3 b3
    const unsigned l0 = (77u * (a & 255u) + 150u * ((a >> 8) & 255u) + 29u * ((a >> 16) & 255u) + 128u) >> 8;
    const unsigned l1 = (77u * (a >> 24) + 150u * (b & 255u) + 29u * ((b >> 8) & 255u) + 128u) >> 8;
    const unsigned l2 = (77u * ((b >> 16) & 255u) + 150u * (b >> 24) + 29u * (c & 255u) + 128u) >> 8;
    const unsigned l3 = (77u * ((c >> 8) & 255u) + 150u * ((c >> 16) & 255u) + 29u * (c >> 24) + 128u) >> 8;
    return l0 | (l1 << 8) | (l2 << 16) | (l3 << 24);
}

__device__ __forceinline__ unsigned luma1(const uint8_t *p, int C)
{
    return C == 1 ? (unsigned)__ldg(p) : (77u * __ldg(p) + 150u * __ldg(p + 1) + 29u * __ldg(p + 2) + 128u) >> 8;
}

// The aligned words of one row that the fast path reads: RGB bytes 3x-4 ..
// 3x+15 (five words), gray bytes x-4 .. x+7 (three).
struct L0Words { unsigned w[5]; };

__device__ __forceinline__ L0Words l0_words(const uint8_t *__restrict__ src, int pitch, int C, int x, int yy)
{
    const uint8_t *row = src + (size_t)yy * pitch;
    const unsigned *q = reinterpret_cast<const unsigned *>(row + C * x) - 1;
    L0Words v;
#pragma unroll
    for (int k = 0; k < 5; ++k) v.w[k] = (C == 3 || k < 3) ? __ldg(q + k) : 0u;
    return v;
}

// Luma of columns x-1 (byte 0 of lo), x..x+3 (mid), x+4 (byte 0 of hi) from a
// row's fast-path words.
__device__ __forceinline__ void luma_words(const L0Words &v, int C, unsigned &lo, unsigned &mid, unsigned &hi)
{
    if (C == 3) {
        const unsigned wl = v.w[0], wr = v.w[4];
        mid = luma4(v.w[1], v.w[2], v.w[3]);
        // x-1: bytes 1..3 of the word before; x+4: bytes 0..2 of the word after
        lo = (77u * ((wl >> 8) & 255u) + 150u * ((wl >> 16) & 255u) + 29u * (wl >> 24) + 128u) >> 8;
        hi = (77u * (wr & 255u) + 150u * ((wr >> 8) & 255u) + 29u * ((wr >> 16) & 255u) + 128u) >> 8;
    } else {
        lo = v.w[0] >> 24;
        mid = v.w[1];
        hi = v.w[2] & 255u;
    }
}

// Luma of columns x-1 (byte 0 of lo), x..x+3 (mid), x+4 (byte 0 of hi) of row yy.
__device__ __forceinline__ void luma_row(const uint8_t *__restrict__ src, int pitch, int C, int w, int x, int yy,
                                        bool fast, unsigned &lo, unsigned &mid, unsigned &hi)
{
    const uint8_t *row = src + (size_t)yy * pitch;
    if (fast) {
        if (C == 3) {
            const unsigned *q = reinterpret_cast<const unsigned *>(row + 3 * x);
            const unsigned wl = __ldg(q - 1), a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), wr = __ldg(q + 3);
            mid = luma4(a, b, c);
            // x-1: bytes 1..3 of the word before; x+4: bytes 0..2 of the word after
            lo = (77u * ((wl >> 8) & 255u) + 150u * ((wl >> 16) & 255u) + 29u * (wl >> 24) + 128u) >> 8;
            hi = (77u * (wr & 255u) + 150u * ((wr >> 8) & 255u) + 29u * ((wr >> 16) & 255u) + 128u) >> 8;
        } else {
            const unsigned *q = reinterpret_cast<const unsigned *>(row + x);
            lo = __ldg(q - 1) >> 24;
            mid = __ldg(q);
            hi = __ldg(q + 1) & 255u;
        }
        return;
    }
    unsigned v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = luma1(row + (size_t)clampi(x - 1 + k, 0, w - 1) * C, C);
    lo = v[0];
    mid = v[1] | (v[2] << 8) | (v[3] << 16) | (v[4] << 24);
    hi = v[5];
}

template <typename PT>
__device__ __forceinline__ void emit_row(const StreamDev &D, int slot, int l, int x, int y, int w, unsigned up,
                                         unsigned lo, unsigned mid, unsigned hi, unsigned dn)
{
    typedef typename Plane2<PT>::type PT2;
    const size_t o = (size_t)y * D.lp[l] + x;
    *reinterpret_cast<unsigned *>(D.u8[slot][l] + o) = mid;
    if constexpr (sizeof(PT) == 2) {
        // FP16: a byte b under the exponent of 1024 is the half 1024 + b (exact,
        // b < 2^10), so one packed subtract gives b itself and the difference
        // of two such halves is exactly the difference of the bytes.
        constexpr unsigned M = 0x64646464u;
        const __half2 k1024 = __half2half2(__ushort_as_half((unsigned short)0x6400u));
        const __half2 half = __half2half2(__ushort_as_half((unsigned short)0x3800u));
        auto h2 = [](unsigned u) { return *reinterpret_cast<const __half2 *>(&u); };
        auto u32 = [](__half2 h) { return *reinterpret_cast<const unsigned *>(&h); };
        uint2 iv;
        iv.x = u32(__hsub2(h2(__byte_perm(mid, M, 0x4140)), k1024));
        iv.y = u32(__hsub2(h2(__byte_perm(mid, M, 0x4342)), k1024));
        *reinterpret_cast<uint2 *>(reinterpret_cast<__half *>(D.pI[slot][l]) + o) = iv;
        // right and left neighbours of columns x .. x+3 (beyond the image edge
        // the last column replicates), paired byte-wise with the rows below / above
        unsigned rt = __byte_perm(mid, hi, 0x4321);
        if (x + 4 > w - 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (x + k + 1 > w - 1) rt = (rt & ~(255u << (8 * k))) | (mid & (255u << (8 * k)));
        }
        const unsigned lf = __byte_perm(mid, lo, 0x2104);
        const unsigned rd01 = __byte_perm(rt, dn, 0x5140), rd23 = __byte_perm(rt, dn, 0x7362);
        const unsigned lu01 = __byte_perm(lf, up, 0x5140), lu23 = __byte_perm(lf, up, 0x7362);
        auto g = [&](unsigned rd, unsigned lu, unsigned sel) {   // (gx, gy) of one pixel
            return u32(__hmul2(__hsub2(h2(__byte_perm(rd, M, sel)), h2(__byte_perm(lu, M, sel))), half));
        };
        uint4 gv;
        gv.x = g(rd01, lu01, 0x4140);
        gv.y = g(rd01, lu01, 0x4342);
        gv.z = g(rd23, lu23, 0x4140);
        gv.w = g(rd23, lu23, 0x4342);
        *reinterpret_cast<uint4 *>(reinterpret_cast<PT2 *>(D.pG[slot][l]) + o) = gv;
    } else {
        const int b[6] = {(int)lo, (int)(mid & 255u), (int)((mid >> 8) & 255u), (int)((mid >> 16) & 255u),
                          (int)(mid >> 24), (int)hi};
        float I[4], gx[4], gy[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // columns beyond the image edge replicate the last column
            const int r = (x + k + 1 <= w - 1) ? b[k + 2] : b[k + 1];
            I[k] = (float)b[k + 1];
            gx[k] = 0.5f * (float)(r - b[k]);
            gy[k] = 0.5f * (float)((int)((dn >> (8 * k)) & 255u) - (int)((up >> (8 * k)) & 255u));
        }
        store_I(reinterpret_cast<PT *>(D.pI[slot][l]) + o, I);
        store_G(reinterpret_cast<PT2 *>(D.pG[slot][l]) + o, gx, gy);
    }
}

template <typename PT>
__global__ void __launch_bounds__(L0_GROUPS) k_level0(const StreamDev *__restrict__ S, WorkList wl, FrameSrc ov)
{
    for (int item = blockIdx.x; item < wl.total; item += gridDim.x) {
        const int s = wl_stream(wl, item);
        const StreamDev &D = S[s];
        const int local = item - __ldg(&wl.prefix[s]);
        const uint8_t *src;
        int pitch, C, slot;
        if (ov.ptr) {
            src = ov.ptr; pitch = ov.pitch; C = ov.channels; slot = ov.slot;
        } else {
            long long t = D.st->t;
            slot = stab_pslot(t);
            src = D.ring + (t % D.ring_len) * D.slot_bytes;
            pitch = D.in_pitch; C = D.C;
        }
        const int w = D.w, h = D.h;
        const int ngx = (w + 4 * L0_GROUPS - 1) / (4 * L0_GROUPS);
        const int x = ((local % ngx) * L0_GROUPS + threadIdx.x) * 4, y0 = (local / ngx) * L0_STRIP;
        if (x >= w) continue;
        // word loads need x-1 .. x+4 inside the row and 4-byte aligned rows
        const bool fast = x >= 4 && x + 8 <= w && ((reinterpret_cast<uintptr_t>(src) | (uintptr_t)pitch) & 3) == 0;
        const int y1 = min(y0 + L0_STRIP, h);
        unsigned plo, pmid, phi, clo, cmid, chi;
        unsigned dummy0, dummy1;
        luma_row(src, pitch, C, w, x, max(y0 - 1, 0), fast, dummy0, pmid, dummy1);
        luma_row(src, pitch, C, w, x, y0, fast, clo, cmid, chi);
        (void)plo; (void)phi;
        // fast path: the words of row y + 2 are in flight while row y + 1's luma
        // and row y's planes are formed
        L0Words nw{};
        if (fast) nw = l0_words(src, pitch, C, x, min(y0 + 1, h - 1));
        for (int y = y0; y < y1; ++y) {
            unsigned nlo, nmid, nhi;
            if (fast) {
                const L0Words cw = nw;
                if (y + 1 < y1) nw = l0_words(src, pitch, C, x, min(y + 2, h - 1));
                luma_words(cw, C, nlo, nmid, nhi);
            } else {
                luma_row(src, pitch, C, w, x, min(y + 1, h - 1), false, nlo, nmid, nhi);
            }
            emit_row<PT>(D, slot, 0, x, y, w, pmid, clo, cmid, chi, nmid);
            pmid = cmid;
            clo = nlo; cmid = nmid; chi = nhi;
        }
    }
}

// Level l >= 1 from level l-1 (REDUCE), as barrier-free strips: a warp owns
// stab_pd_rows output rows of STAB_PD_COLS columns, a thread 4 columns x ..
// x+3, and walks down them.  Per input row it loads the bytes 2x-2 .. 2x+8
// (three aligned loads inside the row; singly with reflect-101 at the row
// ends) and forms the [1 4 6 4 1] row sums of columns 2x, 2x+2, 2x+4, 2x+6 as
// two pairs of 16-bit lanes, so every add and multiply-add serves two outputs
// (a lane's sum is at most 16 * 255 = 4080).  Five such rows give an output row
// the same way (at most 65280 + 128 per lane), rounded and packed to bytes by
// one byte permutation.  An output row is emitted (u8, I, Ix, Iy) once the
// row below it exists; the columns beside a thread's four come from the
// neighbouring lanes, which is why lanes 0 and 31 emit nothing.

// Input bytes 2x-2 .. 2x+8 of one row: wl holds 2x-2, 2x-1 in bytes 2, 3; w0 and
// w1 hold 2x .. 2x+7; wr holds 2x+8 in byte 0.
struct PdWords { unsigned wl, w0, w1, wr; };

__device__ __forceinline__ PdWords pd_words(const uint8_t *__restrict__ row, int x, int wi, bool fast)
{
    PdWords v;
    if (fast) {
        const unsigned *q = reinterpret_cast<const unsigned *>(row + 2 * x);
        const uint2 m = __ldg(reinterpret_cast<const uint2 *>(q));
        v.wl = __ldg(q - 1); v.w0 = m.x; v.w1 = m.y; v.wr = __ldg(q + 2);
    } else {
        unsigned b[11];
#pragma unroll
        for (int k = 0; k < 11; ++k) b[k] = __ldg(row + reflect101(2 * x - 2 + k, wi));
        v.wl = (b[0] << 16) | (b[1] << 24);
        v.w0 = b[2] | (b[3] << 8) | (b[4] << 16) | (b[5] << 24);
        v.w1 = b[6] | (b[7] << 8) | (b[8] << 16) | (b[9] << 24);
        v.wr = b[10];
    }
    return v;
}

// Row sums of columns 2x, 2x+2 (h01: low, high lane) and 2x+4, 2x+6 (h23).
// With b_k the byte at column 2x+k: e0 = (b0, b2), o0 = (b1, b3), e1 = (b4, b6),
// o1 = (b5, b7), and the shifted pairs (b-2, b0), (b-1, b1), (b2, b4), (b3, b5),
// (b6, b8) come from single byte permutations.
__device__ __forceinline__ void pd_hsum(const PdWords &v, unsigned &h01, unsigned &h23)
{
    const unsigned e0 = __byte_perm(v.w0, 0u, 0x4240), o0 = __byte_perm(v.w0, 0u, 0x4341);
    const unsigned e1 = __byte_perm(v.w1, 0u, 0x4240), o1 = __byte_perm(v.w1, 0u, 0x4341);
    const unsigned sl = __byte_perm(v.wl, e0, 0x5452), tl = __byte_perm(v.wl, o0, 0x5453);
    const unsigned sm = __byte_perm(e0, e1, 0x5432), tm = __byte_perm(o0, o1, 0x5432);
    const unsigned sr = __byte_perm(e1, v.wr, 0x3432);
    h01 = sl + 4u * (tl + o0) + 6u * e0 + sm;
    h23 = sm + 4u * (tm + o1) + 6u * e1 + sr;
}

// (sum of [1 4 6 4 1] x five rows of lane pairs + 128) >> 8 for both pairs,
// packed as the bytes of columns x .. x+3.
__device__ __forceinline__ unsigned pd_vsum(unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned a4,
                                            unsigned b0, unsigned b1, unsigned b2, unsigned b3, unsigned b4)
{
    const unsigned va = a0 + a4 + 4u * (a1 + a3) + 6u * a2 + 0x00800080u;
    const unsigned vb = b0 + b4 + 4u * (b1 + b3) + 6u * b2 + 0x00800080u;
    return __byte_perm(va, vb, 0x7531);
}

template <typename PT>
__global__ void __launch_bounds__(128) k_pyr_down(const StreamDev *__restrict__ S, WorkList wl, int l, int slot_ov)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < wl.total; item += nwarps) {
        const int s = wl_stream(wl, item);
        const StreamDev &D = S[s];
        const int local = item - __ldg(&wl.prefix[s]);
        const int slot = slot_ov >= 0 ? slot_ov : stab_pslot(D.st->t);
        const uint8_t *in = D.u8[slot][l - 1];
        const int wi = D.lw[l - 1], hi = D.lh[l - 1], pi = D.lp[l - 1];
        const int wo = D.lw[l], ho = D.lh[l];
        const int ncx = (wo + STAB_PD_COLS - 1) / STAB_PD_COLS, R = stab_pd_rows(ho);
        const int x = (local % ncx) * STAB_PD_COLS + 4 * (lane - 1), y0 = (local / ncx) * R;
        const int y1 = min(y0 + R, ho);
        // bytes 2x-4 .. 2x+11 lie inside the padded row and 2x-2 .. 2x+8 inside the image row
        const bool fast = x >= 4 && 2 * x + 8 <= wi - 1 && 2 * x + 12 <= pi;
        auto words = [&](int yy) { return pd_words(in + (size_t)reflect101(yy, hi) * pi, x, wi, fast); };
        // row sums of input rows 2r-2, 2r-1, 2r, where r is the next output row
        int r = max(y0 - 1, 0);
        unsigned a0, b0, a1, b1, a2, b2;
        pd_hsum(words(2 * r - 2), a0, b0);
        pd_hsum(words(2 * r - 1), a1, b1);
        pd_hsum(words(2 * r), a2, b2);
        auto next_row = [&]() -> unsigned {
            unsigned a3, b3, a4, b4;
            pd_hsum(words(2 * r + 1), a3, b3);
            pd_hsum(words(2 * r + 2), a4, b4);
            const unsigned o = pd_vsum(a0, a1, a2, a3, a4, b0, b1, b2, b3, b4);
            a0 = a2; b0 = b2; a1 = a3; b1 = b3; a2 = a4; b2 = b4;
            ++r;
            return o;
        };
        // rows y-1, y (replicated above row 0) and y+1 (replicated below row ho-1)
        unsigned up = next_row();
        unsigned mid = y0 == 0 ? up : next_row();
        for (int y = y0; y < y1; ++y) {
            const unsigned dn = y + 1 <= ho - 1 ? next_row() : mid;
            unsigned lo = __shfl_up_sync(0xffffffffu, mid, 1) >> 24;
            const unsigned hb = __shfl_down_sync(0xffffffffu, mid, 1) & 255u;
            if (x == 0) lo = mid & 255u;   // replicated left border
            if (lane >= 1 && lane <= 30 && x < wo) emit_row<PT>(D, slot, l, x, y, wo, up, lo, mid, hb, dn);
            up = mid;
            mid = dn;
        }
    }
}

// Levels l0 .. l0 + D - 1 (D <= 3) of a stream in one launch, from level
// l0 - 1 in global memory.  A block owns a PT_TH x PT_TW tile of the stream's
// last fused level lt = l0 + D - 1 and the tiles 2^k times larger of level
// lt - k.  It stages the rows and columns of level l0 - 1 those tiles need
// (their own pixels, the halos of the later levels and the neighbours of the
// planes) into shared memory with 16-byte cp.async, then builds each fused
// level's region in shared memory from the region of the level above it
// (the same packed 16-bit REDUCE sums as the strip kernel), and emits each
// level's own tile (u8, I, Ix, Iy).  Out-of-image taps are reflect-101
// indices into the level above, so every region only ever holds pixels of the
// image; the regions of the levels are derived from the last one:
//   B0 (level lt): rows [Y0 - 1, Y1 + 1), columns [X0 - 4, X1 + 1) (quads)
//   B(k+1): rows [2 ys_k - 2, 2 ye_k + 1), columns [2 xs_k - 4, 2 xe_k + 4)
// which covers the five-tap inputs of every quad of B(k) and the one-pixel
// neighbourhood of level k + 1's own tile.
constexpr int PT_TH = 8, PT_TW = 32, PT_THREADS = 256, PT_MAXD = 3;

struct PtRegion {
    int ys, ye, xs, xe;   // rows [ys, ye), columns [xs, xe) of the level (unclipped); xs % 4 == 0
    int stride;           // bytes per buffer row
    int off;              // byte offset of the buffer in shared memory
};

// Regions and buffer offsets of a tile whose last level's tile starts at
// (X0, Y0); k = 0 is the last fused level, k = D the staged input level.
__host__ __device__ inline int pt_regions(int D, int X0, int Y0, int X1, int Y1, PtRegion *R)
{
    R[0].ys = Y0 - 1; R[0].ye = Y1 + 1;
    R[0].xs = (X0 - 4) & ~3;
    R[0].xe = (X1 + 1 + 3) & ~3;
    for (int k = 0; k < D; ++k) {
        R[k + 1].ys = 2 * R[k].ys - 2;
        R[k + 1].ye = 2 * R[k].ye + 1;
        R[k + 1].xs = 2 * R[k].xs - 4;
        R[k + 1].xe = 2 * R[k].xe + 4;
    }
    // the staged level starts on a 16-byte column for the copies
    R[D].xs = R[D].xs & ~15;
    int off = 0;
    for (int k = 0; k <= D; ++k) {
        R[k].stride = ((R[k].xe - R[k].xs) + 8 + 15) & ~15;   // + the hi byte and a word of slack
        R[k].off = off;
        off += R[k].stride * (R[k].ye - R[k].ys);
    }
    return off;
}

// Largest shared-memory footprint of a tile (interior tile, D = PT_MAXD).
__host__ __device__ inline int pt_smem_bytes()
{
    PtRegion R[PT_MAXD + 1];
    return pt_regions(PT_MAXD, 64, 64, 64 + PT_TW, 64 + PT_TH, R) + 64;
}

// Walks e = first, first + PT_THREADS, ... over n items of rows of `per`
// items as (row, column) pairs without a division per step.
struct PtWalk {
    int r, c, dr, dc, per;
    __device__ PtWalk(int first, int per_) : per(per_)
    {
        r = first / per; c = first - r * per;
        dr = PT_THREADS / per; dc = PT_THREADS - dr * per;
    }
    __device__ void next()
    {
        r += dr; c += dc;
        if (c >= per) { c -= per; ++r; }
    }
};

// REDUCE sums of the five-tap row of input row gy for the quad at column x
// (packed 16-bit lanes, see pd_hsum); `fast` quads read four aligned words.
__device__ __forceinline__ void pt_hrow(const unsigned char *row, int x, int wi, int xs, bool fast, unsigned &a,
                                        unsigned &b)
{
    PdWords v;
    if (fast) {
        const unsigned *q = reinterpret_cast<const unsigned *>(row + (2 * x - 4 - xs));
        v.wl = q[0]; v.w0 = q[1]; v.w1 = q[2]; v.wr = q[3];
    } else {
        unsigned bb[11];
#pragma unroll
        for (int i = 0; i < 11; ++i) bb[i] = row[reflect101(2 * x - 2 + i, wi) - xs];
        v.wl = (bb[0] << 16) | (bb[1] << 24);
        v.w0 = bb[2] | (bb[3] << 8) | (bb[4] << 16) | (bb[5] << 24);
        v.w1 = bb[6] | (bb[7] << 8) | (bb[8] << 16) | (bb[9] << 24);
        v.wr = bb[10];
    }
    pd_hsum(v, a, b);
}

template <typename PT>
__global__ void __launch_bounds__(PT_THREADS, 4) k_pyr_tail(const StreamDev *__restrict__ S, WorkList wl, int l0,
                                                         int l1, int slot_ov)
{
    extern __shared__ __align__(16) unsigned char pt_smem[];
    __shared__ PtRegion sreg[PT_MAXD + 1];
    const int tid = threadIdx.x;
    for (int item = blockIdx.x; item < wl.total; item += gridDim.x) {
        const int s = wl_stream(wl, item);
        const StreamDev &D = S[s];
        const int local = item - __ldg(&wl.prefix[s]);
        const int slot = slot_ov >= 0 ? slot_ov : stab_pslot(D.st->t);
        const int lt = min(l1, D.L) - 1, nd = lt - l0 + 1;   // fused levels of this stream
        const int ntx = (D.lw[lt] + PT_TW - 1) / PT_TW;
        const int X0 = (local % ntx) * PT_TW, Y0 = (local / ntx) * PT_TH;
        if (tid == 0) pt_regions(nd, X0, Y0, X0 + PT_TW, Y0 + PT_TH, sreg);
        __syncthreads();
        // ---- stage level l0 - 1: the clipped region, whole 16-byte chunks of the rows
        {
            const int li = l0 - 1, wi = D.lw[li], hi = D.lh[li], pi = D.lp[li];
            const PtRegion Q = sreg[nd];
            const int r0 = max(Q.ys, 0), r1 = min(Q.ye, hi);
            const int c0 = max(Q.xs, 0), c1 = min(Q.xe, wi);   // c0 % 16 == 0
            const int nch = c1 > c0 ? (c1 - c0 + 15) >> 4 : 0, n = (r1 - r0) * nch;
            const uint8_t *src = D.u8[slot][li];
            unsigned char *dst = pt_smem + Q.off;
            if (n > 0) {
                PtWalk wk(tid, nch);
                for (int e = tid; e < n; e += PT_THREADS, wk.next()) {
                    const int gy = r0 + wk.r, gx = c0 + 16 * wk.c;   // gx + 16 <= pitch: the chunk stays in the row
                    const unsigned d =
                        (unsigned)__cvta_generic_to_shared(dst + (gy - Q.ys) * Q.stride + (gx - Q.xs));
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d),
                                 "l"(src + (size_t)gy * pi + gx) : "memory");
                }
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncthreads();
        }
        // ---- levels l0 .. lt: build region k from region k + 1, emit the tile of k + 1
        for (int k = nd - 1; k >= -1; --k) {
            // emit the own tile of the level of region k + 1 (if it is a fused level)
            if (k + 1 < nd) {
                const int l = lt - (k + 1);
                const int w = D.lw[l], h = D.lh[l];
                const PtRegion Q = sreg[k + 1];
                const unsigned char *b = pt_smem + Q.off;
                const int oy0 = Y0 << (k + 1), oy1 = min((Y0 + PT_TH) << (k + 1), h);
                const int ox0 = X0 << (k + 1), ox1 = min((X0 + PT_TW) << (k + 1), w);
                const int nq = (ox1 - ox0 + 3) >> 2, n = (oy1 - oy0) * nq;
                if (n > 0) {
                    PtWalk wk(tid, nq);
                    for (int e = tid; e < n; e += PT_THREADS, wk.next()) {
                        const int x = ox0 + 4 * wk.c, y = oy0 + wk.r;
                        const unsigned char *row = b + (y - Q.ys) * Q.stride + (x - Q.xs);
                        const unsigned mid = *reinterpret_cast<const unsigned *>(row);
                        const unsigned up = y > 0 ? *reinterpret_cast<const unsigned *>(row - Q.stride) : mid;
                        const unsigned dn = y + 1 < h ? *reinterpret_cast<const unsigned *>(row + Q.stride) : mid;
                        const unsigned lo = x > 0 ? row[-1] : (mid & 255u);
                        emit_row<PT>(D, slot, l, x, y, w, up, lo, mid, row[4], dn);
                    }
                }
            }
            if (k < 0) break;
            // build region k (level lt - k) from region k + 1 (level lt - k - 1): a
            // thread walks a band of rows down one quad column, five input row sums in
            // flight (two new ones per output row)
            {
                const int l = lt - k, li = l - 1;
                const int w = D.lw[l], h = D.lh[l], wi = D.lw[li], hi = D.lh[li];
                const PtRegion Q = sreg[k], P = sreg[k + 1];
                const unsigned char *bi = pt_smem + P.off;
                unsigned char *bo = pt_smem + Q.off;
                const int r0 = max(Q.ys, 0), r1 = min(Q.ye, h);
                const int x0 = max(Q.xs, 0), x1 = min(Q.xe, w);
                const int nq = x1 > x0 ? (x1 - x0 + 3) >> 2 : 0, nr = r1 - r0;
                if (nq > 0 && nr > 0) {
                    const int nb = min(max(PT_THREADS / nq, 1), nr);          // bands
                    const int bh = (nr + nb - 1) / nb;                          // rows per band
                    for (int task = tid; task < nq * nb; task += PT_THREADS) {
                        const int band = task / nq, x = x0 + 4 * (task - band * nq);
                        const int ya = r0 + band * bh, yb = min(ya + bh, r1);
                        if (ya >= yb) continue;
                        const bool fast = x >= 1 && 2 * x + 8 <= wi - 1;
                        auto hrow = [&](int v, unsigned &a, unsigned &c) {
                            pt_hrow(bi + (reflect101(v, hi) - P.ys) * P.stride, x, wi, P.xs, fast, a, c);
                        };
                        unsigned a0, c0, a1, c1, a2, c2;
                        hrow(2 * ya - 2, a0, c0);
                        hrow(2 * ya - 1, a1, c1);
                        hrow(2 * ya, a2, c2);
                        unsigned char *o = bo + (ya - Q.ys) * Q.stride + (x - Q.xs);
                        for (int y = ya; y < yb; ++y, o += Q.stride) {
                            unsigned a3, c3, a4, c4;
                            hrow(2 * y + 1, a3, c3);
                            hrow(2 * y + 2, a4, c4);
                            *reinterpret_cast<unsigned *>(o) = pd_vsum(a0, a1, a2, a3, a4, c0, c1, c2, c3, c4);
                            a0 = a2; c0 = c2; a1 = a3; c1 = c3; a2 = a4; c2 = c4;
                        }
                    }
                }
            }
            __syncthreads();
        }
        __syncthreads();   // the buffers and the region table are refilled for the next item
    }
}

template <typename PT>
__global__ void k_plane_f32(const StreamDev *__restrict__ S, int slot, int l, float *I, float *Ix, float *Iy)
{
    typedef typename Plane2<PT>::type PT2;
    const StreamDev &D = S[0];
    const int w = D.lw[l], h = D.lh[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w * h; i += gridDim.x * blockDim.x) {
        int y = i / w, x = i - y * w;
        size_t o = (size_t)y * D.lp[l] + x;
        if (I) I[i] = ld1(reinterpret_cast<const PT *>(D.pI[slot][l]) + o);
        float2 g = ld2(reinterpret_cast<const PT2 *>(D.pG[slot][l]) + o);
        if (Ix) Ix[i] = g.x;
        if (Iy) Iy[i] = g.y;
    }
}

}  // namespace

void launch_level0(const Launch &L, int prec, const StreamDev *S, WorkList wl, FrameSrc ov)
{
    int g = grid_for(L, wl.total, prec ? occ_level0_h() : occ_level0_f());
    if (prec) k_level0<__half><<<g, L0_GROUPS, 0, L.stream>>>(S, wl, ov);
    else k_level0<float><<<g, L0_GROUPS, 0, L.stream>>>(S, wl, ov);
}

void launch_pyr_down(const Launch &L, int prec, const StreamDev *S, WorkList wl, int l, int slot_ov)
{
    // one warp per strip, four warps per block
    int g = grid_for(L, (wl.total + 3) / 4, prec ? occ_pyr_h() : occ_pyr_f());
    if (prec) k_pyr_down<__half><<<g, 128, 0, L.stream>>>(S, wl, l, slot_ov);
    else k_pyr_down<float><<<g, 128, 0, L.stream>>>(S, wl, l, slot_ov);
}

static int occ_tail(int prec)
{
    static DevCache c[2];
    return c[prec ? 1 : 0].get([prec] {
        int v = 0;
        const int smem = pt_smem_bytes();
        cudaError_t e;
        if (prec) {
            cudaFuncSetAttribute(k_pyr_tail<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_pyr_tail<__half>, PT_THREADS, smem);
        } else {
            cudaFuncSetAttribute(k_pyr_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_pyr_tail<float>, PT_THREADS, smem);
        }
        return (e != cudaSuccess || v < 1) ? 1 : v;
    });
}

int pyr_tail_tile_w() { return PT_TW; }
int pyr_tail_tile_h() { return PT_TH; }
int pyr_tail_levels() { return PT_MAXD; }
void warm_pyr_tail() { occ_tail(0); occ_tail(1); }

void launch_pyr_tail(const Launch &L, int prec, const StreamDev *S, WorkList wl, int l0, int l1, int slot_ov)
{
    const int g = grid_for(L, wl.total, occ_tail(prec)), smem = pt_smem_bytes();
    if (prec) k_pyr_tail<__half><<<g, PT_THREADS, smem, L.stream>>>(S, wl, l0, l1, slot_ov);
    else k_pyr_tail<float><<<g, PT_THREADS, smem, L.stream>>>(S, wl, l0, l1, slot_ov);
}

void launch_plane_f32(const Launch &L, int prec, const StreamDev *S, int slot, int l, float *I, float *Ix, float *Iy)
{
    if (prec) k_plane_f32<__half><<<4 * L.sms, 256, 0, L.stream>>>(S, slot, l, I, Ix, Iy);
    else k_plane_f32<float><<<4 * L.sms, 256, 0, L.stream>>>(S, slot, l, I, Ix, Iy);
}

#define OCC_FN128(name, kern)                                                                  \
    int name()                                                                                 \
    {                                                                                          \
        static DevCache c;                                                                     \
        return c.get([] {                                                                      \
            int v = 0;                                                                         \
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, L0_GROUPS, 0) != cudaSuccess || v < 1) \
                v = 1;                                                                         \
            return v;                                                                          \
        });                                                                                    \
    }
OCC_FN128(occ_level0_f, k_level0<float>)
OCC_FN128(occ_level0_h, k_level0<__half>)
OCC_FN128(occ_pyr_f, k_pyr_down<float>)
OCC_FN128(occ_pyr_h, k_pyr_down<__half>)

// k_lk.cu -- pyramidal Lucas-Kanade (Sec. 3.2, Eq. 3-6; coarse-to-fine as in
// Bouguet's pyramidal implementation cited there) with the forward-backward
// check of Sec. 4.1.
//
// A group of WPF warps (WPF = 1 or 2, chosen by the autotuner) tracks one
// feature.  At each level the group stages the (2r+2)^2 patch of I and of
// (Ix, Iy) under the window into shared memory (asynchronous 8 / 16-byte
// cp.async row copies in the planes' own precision, all of a level's copies in
// flight together; border taps replicated, so sampling is branch-free; FP16
// values widen exactly to FP32 when read), samples the (2r+1)^2
// template bilinearly with weights shared by every sample, and keeps T, Tx,
// Ty in registers (NS samples per thread).  The next frame's patch is staged
// once per level around the initial guess with a small margin, so iterations
// read shared memory only (a larger move re-stages it); each iteration
// accumulates b = sum e [Tx, Ty] and solves the 2x2 system.  Sums are reduced with xor-butterfly shuffles (same
// bits in every lane) and, for two warps, combined through shared memory in a
// fixed order, so every thread of the group takes the same branch.
#include <cuda.h>   // CUtensorMap and the types of its encoding call (no driver library is linked)

#include <cstring>
#include <vector>

#include "kernels.cuh"

namespace {

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Synchronise the threads of one feature group.
template <int WPF>
__device__ __forceinline__ void group_sync(int grp)
{
    if (WPF == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(32 * WPF) : "memory");
}

// Group-wide sums of three values (fixed order: warp 0 + warp 1).
template <int WPF>
__device__ __forceinline__ void group_sum3(float &a, float &b, float &c, float *red, int wig, int grp)
{
    a = wsum(a); b = wsum(b); c = wsum(c);
    if (WPF > 1) {
        const int lane = threadIdx.x & 31;
        group_sync<WPF>(grp);   // previous readers of red are done
        if (lane == 0) { red[3 * wig] = a; red[3 * wig + 1] = b; red[3 * wig + 2] = c; }
        group_sync<WPF>(grp);
        a = red[0]; b = red[1]; c = red[2];
#pragma unroll
        for (int w = 1; w < WPF; ++w) { a += red[3 * w]; b += red[3 * w + 1]; c += red[3 * w + 2]; }
    }
}

// Shared-memory row stride for a patch of width pwid staged from a 4-aligned
// start column (up to 3 extra leading columns, whole 4-element vectors).
__host__ __device__ constexpr int lk_sw(int pwid) { return ((pwid + 6) / 4) * 4; }

template <int BYTES>
__device__ __forceinline__ void cpa(void *sdst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    if (BYTES == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Tensor-memory-access (TMA) staging of the fixed 21 x 21 window's patches.
// A patch lying inside its level is copied by three 2-D tensor copies (the
// template's I and (Ix, Iy) boxes, the next frame's I box) that one lane
// issues, completing on the group's mbarrier; shared rows are the boxes' rows.
// Box columns start at the patch's first column rounded down to 16 bytes
// (the copy's coordinate rule), so a box is A - 1 columns wider than the patch.
template <typename PT>
struct LkTma {
    static constexpr int ES = (int)sizeof(PT), A = 16 / ES;   // column alignment of a box start, elements
    static constexpr int PW = 22, PJ = 26;                     // template and next-frame patch sides
    static constexpr int BWI = (PW + 2 * A - 2) / A * A, BWJ = (PJ + 2 * A - 2) / A * A;
    static constexpr unsigned TX_I = PW * BWI * ES, TX_G = PW * BWI * 2 * ES, TX_J = PJ * BWJ * ES;
    static constexpr int al128(unsigned b) { return (int)((b + 127) / 128 * 128); }
    static constexpr int OFF_G = al128(TX_I), OFF_J = OFF_G + al128(TX_G), OFF_RED = OFF_J + al128(TX_J);
    static constexpr int GROUP = OFF_RED + 128;   // 32 reduction bytes, the mbarrier at +64
    static_assert(BWI * ES % 16 == 0 && BWJ * ES % 16 == 0 && BWI >= PW + A - 1 && BWJ >= PJ + A - 1, "box geometry");
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *mb)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mb)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const void *map, int x, int y, unsigned long long *mb)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(mb))
        : "memory");
}
// Generic-proxy reads of a buffer are ordered before the tensor copies that refill it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// Wait for the mbarrier phase `ph` to complete, giving up after about a second
// of polling (each try_wait suspends briefly); false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long *mb, unsigned ph)
{
    for (int i = 0; i < (1 << 20); ++i) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(mb)), "r"(ph)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// 4 consecutive plane elements (one staged vector) by asynchronous copy.
__device__ __forceinline__ void cpa_vec4(float *d, const float *g) { cpa<16>(d, g); }
__device__ __forceinline__ void cpa_vec4(__half *d, const __half *g) { cpa<8>(d, g); }
__device__ __forceinline__ void cpa_vec4(float2 *d, const float2 *g) { cpa<16>(d, g); cpa<16>(d + 2, g + 2); }
__device__ __forceinline__ void cpa_vec4(__half2 *d, const __half2 *g) { cpa<16>(d, g); }

// Plane elements read from shared memory, widened to FP32 (exact).
__device__ __forceinline__ float f1(float v) { return v; }
__device__ __forceinline__ float f1(__half v) { return __half2float(v); }
__device__ __forceinline__ float2 f2(float2 v) { return v; }
__device__ __forceinline__ float2 f2(__half2 v) { return __half22float2(v); }

// Stage the pwid x pwid patch with top-left (x0, y0) of a plane (element
// type E: the plane's own precision) into shared memory, row stride sw.
// Inside the image, rows are copied asynchronously as aligned 4-element
// vectors from x0 rounded down to a multiple of 4, and the returned column
// offset (x0 - that start) locates the patch; the caller waits for the copies
// (cpa_wait_all) before the group barrier.  Near a border every tap is
// clamped (replicated border) and copied singly, offset 0.
template <typename E, int NT>
__device__ __forceinline__ int stage(const E *__restrict__ P, int pitch, int wl, int hl, int x0, int y0, int pwid,
                                     int sw, bool inside, E *dst, int tig)
{
    const int x0a = x0 & ~3, off = x0 - x0a;
    const int nv = (pwid + off + 3) >> 2;
    if (inside && x0a + 4 * nv <= pitch) {
        const int n = pwid * nv, q = NT / nv, rr = NT - q * nv;
        int row = tig / nv, v = tig - row * nv;
        for (int e = tig; e < n; e += NT) {
            cpa_vec4(dst + row * sw + 4 * v, P + (size_t)(y0 + row) * pitch + x0a + 4 * v);
            v += rr; row += q;
            if (v >= nv) { v -= nv; ++row; }
        }
        return off;
    }
    const int n = pwid * pwid, q = NT / pwid, rr = NT - q * pwid;
    int row = tig / pwid, col = tig - row * pwid;
    for (int e = tig; e < n; e += NT) {
        const int xx = clampi(x0 + col, 0, wl - 1), yy = clampi(y0 + row, 0, hl - 1);
        dst[row * sw + col] = P[(size_t)yy * pitch + xx];
        col += rr; row += q;
        if (col >= pwid) { col -= pwid; ++row; }
    }
    return 0;
}

// The same staging for a PW x PW patch of compile-time size (the fixed-radius
// trackers), cheaper to issue: when the patch's columns lie inside the row,
// every row is copied as NV = (PW + 6) / 4 aligned vectors (covering any
// start offset; the extra vector lies inside the row pitch and is not read),
// lane tig owns vector tig % NV of rows tig / NV, + NT / NV, ... (all index
// arithmetic by constants), and a row outside the plane is replaced by the
// nearest border row (the replicated border).  Otherwise every tap is clamped
// and copied singly, offset 0.
template <typename E, int NT, int PW, int SW>
__device__ __forceinline__ int stage_k(const E *__restrict__ P, int pitch, int wl, int hl, int x0, int y0, E *dst,
                                       int tig)
{
    constexpr int NV = (PW + 6) / 4, RPP = NT / NV, NPASS = (PW + RPP - 1) / RPP;
    static_assert(4 * NV <= SW && RPP >= 1, "a staged row fits the stride");
    const int x0a = x0 & ~3;
    if (x0 >= 0 && x0 + PW <= wl && x0a + 4 * NV <= pitch) {
        const int v = tig % NV, r0 = tig / NV;
        if (r0 < RPP) {
            const E *src = P + x0a + 4 * v;
            E *d = dst + 4 * v;
            const bool rows_in = y0 >= 0 && y0 + PW <= hl;
#pragma unroll
            for (int i = 0; i < NPASS; ++i) {
                const int r = r0 + RPP * i;
                if (r < PW) {
                    const int yy = rows_in ? y0 + r : clampi(y0 + r, 0, hl - 1);
                    cpa_vec4(d + r * SW, src + (size_t)yy * pitch);
                }
            }
        }
        return x0 - x0a;
    }
    constexpr int n = PW * PW, q = NT / PW, rr = NT - q * PW;
    int row = tig / PW, col = tig - row * PW;
    for (int e = tig; e < n; e += NT) {
        const int xx = clampi(x0 + col, 0, wl - 1), yy = clampi(y0 + row, 0, hl - 1);
        dst[row * SW + col] = P[(size_t)yy * pitch + xx];
        col += rr; row += q;
        if (col >= PW) { col -= PW; ++row; }
    }
    return 0;
}

// Margin (px) of the next frame's staged patch: iterations whose window stays
// within it sample shared memory only; a larger move re-stages the patch.
constexpr int LK_MARGIN = 2;

// Samples per column segment for NS samples per thread (segments of 7 rows
// for the 21 x 21 window and smaller, of 5 rows for radius 11 and 12).
__host__ __device__ constexpr int lk_seg(int ns) { return ns % 7 == 0 ? 7 : 5; }

// Bilinear sampling shared by the template and the iterations: a thread walks
// column segments of the window (segment s: column s % ww, rows
// SEG (s / ww) .. + SEG - 1), forming the horizontal lerp of each patch row
// once and one vertical lerp per sample, so a segment of SEG samples reads
// SEG + 1 rows of two taps.
__device__ __forceinline__ float lerpf(float a, float b, float f) { return fmaf(f, b - a, a); }

// Track one feature from pyramid slot sa to slot sb.  RC = compile-time
// radius (0: runtime D.r).  sI: pw rows of I, sG: pw rows of (Ix, Iy), sJ:
// pw + 2 LK_MARGIN rows of the next frame's I (plane precision), red: 3 * WPF.
// TS: the template (T, Tx, Ty per sample pair) lives in shared memory at sT
// (3 NS / 2 packed pairs per thread, thread-interleaved so a warp's accesses
// are conflict-free) instead of 3 NS registers, for a register budget that
// lets more warps reside; otherwise sT is unused.
// Not inlined: the kernel calls it for the forward and the backward track, and
// one copy of its unrolled body keeps the instruction working set small.
// TM: patches lying inside their level are copied by tensor copies (LkTma),
// the rest by stage_k into the same layout; mb / ph: the group's mbarrier and
// its phase.
template <typename PT, int NS, int RC, int WPF, bool TS, bool TM>
__device__ __noinline__ bool lk_track(const StreamDev &D, int sa, int sb, float ux, float uy, float &vx, float &vy, int &iters,
                         int &tpl, PT *sI, typename Plane2<PT>::type *sG, PT *sJ, float *red, fx2 *sT,
                         unsigned long long *mb, unsigned &ph, int tig, int grp)
{
    static_assert(!TM || (RC == 10 && WPF == 1 && !TS), "tensor-copy staging serves the 21 x 21 window, one warp");
    typedef LkTma<PT> TG;
    typedef typename Plane2<PT>::type PT2;
    constexpr int NT = 32 * WPF;
    const int wig = tig >> 5;
    const int r = RC ? RC : D.r, ww = 2 * r + 1, pw = ww + 1, N = ww * ww;
    const int pj = pw + 2 * LK_MARGIN;
    const int swI = TM ? TG::BWI : lk_sw(pw), swJ = TM ? TG::BWJ : lk_sw(pj);
    constexpr int SEG = lk_seg(NS), Q = NS / SEG;
    // EXACT: segments tile the window's rows exactly, so every row a segment
    // reads (its SEG + 1 rows) lies in the patch and needs no clamp; a thread
    // without a segment reads rows 0 .. SEG (finite, staged) with weight 0.
    constexpr bool EXACT = RC > 0 && (2 * RC + 1) % SEG == 0;
    const int nseg = (ww + SEG - 1) / SEG;
    int scol[Q], srow[Q];   // this thread's segments (sv false: none)
    bool sv[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int sgi = tig + NT * q;
        sv[q] = sgi < ww * nseg;
        scol[q] = sgi % ww;
        srow[q] = sv[q] ? (sgi / ww) * SEG : (EXACT ? 0 : ww);
    }
    // row k of segment q (k = 0 .. SEG) and whether its sample e lies in the window
    auto srw = [&](int q, int k) { return EXACT ? srow[q] + k : min(srow[q] + k, pw - 1); };
    auto sok = [&](int q, int e) { return EXACT ? sv[q] : srow[q] + e < ww; };
    float gx = 0.f, gy = 0.f, dx = 0.f, dy = 0.f;
    // An even number of segments per thread runs as pairs (segments 2p, 2p+1
    // in the two lanes of packed f32x2 arithmetic); T, Tx, Ty are kept as pairs.
    constexpr bool PAIR = Q % 2 == 0;
    constexpr int NP = PAIR ? NS / 2 : 1;
    static_assert(!TS || (PAIR && WPF == 1), "the shared template is laid out for pairs and one warp");
    float T[PAIR ? 1 : NS], TX[PAIR ? 1 : NS], TY[PAIR ? 1 : NS];
    fx2 TT[(PAIR && !TS) ? NP : 1], TTX[(PAIR && !TS) ? NP : 1], TTY[(PAIR && !TS) ? NP : 1];
    // template pair m, component k (0: T, 1: Tx, 2: Ty) of this thread
    auto tref = [&](int m, int k) -> fx2 & {
        if constexpr (TS) return sT[(3 * m + k) * 32 + tig];
        else return k == 0 ? TT[m] : (k == 1 ? TTX[m] : TTY[m]);
    };
    // EXACT windows: a segment without samples (past the window) still reads
    // staged, finite values, so its samples are not masked one by one; its
    // lane's share of every sum (G and b) is dropped once, after accumulating.
    constexpr bool MASK_END = EXACT && Q == 2;
    auto psum = [&](fx2 v, int pp) {
        float u0, u1;
        upk(v, u0, u1);
        if constexpr (MASK_END) return (sv[2 * pp] ? u0 : 0.f) + (sv[2 * pp + 1] ? u1 : 0.f);
        else return u0 + u1;
    };
    for (int l = D.L - 1; l >= 0; --l) {
        const PT *Ia = reinterpret_cast<const PT *>(D.pI[sa][l]);
        const PT2 *Ga = reinterpret_cast<const PT2 *>(D.pG[sa][l]);
        const PT *Jb = reinterpret_cast<const PT *>(D.pI[sb][l]);
        const int wl = D.lw[l], hl = D.lh[l], p = D.lp[l];
        const float sc = __int_as_float((127 - l) << 23);   // 2^-l
        const float px = ux * sc, py = uy * sc;
        const float bx = fminf(fmaxf(px, -64.f), (float)wl + 64.f);
        const float by = fminf(fmaxf(py, -64.f), (float)hl + 64.f);
        const float fx = floorf(bx), fy = floorf(by);
        const float ax = bx - fx, ay = by - fy;
        const int ix = (int)fx - r, iy = (int)fy - r;
        const bool inside = ix >= 0 && ix + ww <= wl - 1 && iy >= 0 && iy + ww <= hl - 1;
        // next frame's patch around the level's initial guess, with a margin
        int jx0 = (int)floorf(fminf(fmaxf(px + gx, -64.f), (float)wl + 64.f)) - r - LK_MARGIN;
        int jy0 = (int)floorf(fminf(fmaxf(py + gy, -64.f), (float)hl + 64.f)) - r - LK_MARGIN;
        bool jin = jx0 >= 0 && jx0 + pj - 1 <= wl - 1 && jy0 >= 0 && jy0 + pj - 1 <= hl - 1;
        group_sync<WPF>(grp);
        int offI, offJ;
        if constexpr (TM) {
            const unsigned char *maps = static_cast<const unsigned char *>(D.tmap);
            const bool tin = maps && ix >= 0 && ix + TG::PW <= wl && iy >= 0 && iy + TG::PW <= hl && jx0 >= 0 &&
                             jx0 + TG::PJ <= wl && jy0 >= 0 && jy0 + TG::PJ <= hl;
            if (tin) {
                const int xa = ix & ~(TG::A - 1), jxa = jx0 & ~(TG::A - 1);
                offI = ix - xa;
                offJ = jx0 - jxa;
                if (tig == 0) {
                    const unsigned char *mt = maps + (size_t)((sa * STAB_MAXL + l) * 3) * 128;
                    const unsigned char *mj = maps + (size_t)((sb * STAB_MAXL + l) * 3 + 2) * 128;
                    fence_proxy_async();
                    mbar_expect_tx(mb, TG::TX_I + TG::TX_G + TG::TX_J);
                    tma_load_2d(sI, mt, xa, iy, mb);
                    tma_load_2d(sG, mt + 128, xa, iy, mb);
                    tma_load_2d(sJ, mj, jxa, jy0, mb);
                }
                if (!mbar_wait(mb, ph)) set_err(D.st, STAB_ERR_TIMEOUT);
                ph ^= 1u;
            } else {
                offI = stage_k<PT, NT, TG::PW, TG::BWI>(Ia, p, wl, hl, ix, iy, sI, tig);
                stage_k<PT2, NT, TG::PW, TG::BWI>(Ga, p, wl, hl, ix, iy, sG, tig);
                offJ = stage_k<PT, NT, TG::PJ, TG::BWJ>(Jb, p, wl, hl, jx0, jy0, sJ, tig);
            }
        } else if constexpr (RC > 0) {
            constexpr int PWc = 2 * RC + 2, PJc = PWc + 2 * LK_MARGIN, SWI = lk_sw(PWc), SWJ = lk_sw(PJc);
            offI = stage_k<PT, NT, PWc, SWI>(Ia, p, wl, hl, ix, iy, sI, tig);
            stage_k<PT2, NT, PWc, SWI>(Ga, p, wl, hl, ix, iy, sG, tig);
            offJ = stage_k<PT, NT, PJc, SWJ>(Jb, p, wl, hl, jx0, jy0, sJ, tig);
        } else {
            offI = stage<PT, NT>(Ia, p, wl, hl, ix, iy, pw, swI, inside, sI, tig);
            stage<PT2, NT>(Ga, p, wl, hl, ix, iy, pw, swI, inside, sG, tig);
            offJ = stage<PT, NT>(Jb, p, wl, hl, jx0, jy0, pj, swJ, jin, sJ, tig);
        }
        cpa_wait_all();
        group_sync<WPF>(grp);
        float gxx = 0.f, gxy = 0.f, gyy = 0.f;
        if constexpr (PAIR) {
            const fx2 AX = pk(ax, ax), AY = pk(ay, ay);
            fx2 sxx = pk(0.f, 0.f), sxy = sxx, syy = sxx;
#pragma unroll
            for (int pp = 0; pp < Q / 2; ++pp) {
                const int qa = 2 * pp, qb = 2 * pp + 1;
                const PT *pIa = sI + offI + scol[qa], *pIb = sI + offI + scol[qb];
                const PT2 *pGa = sG + offI + scol[qa], *pGb = sG + offI + scol[qb];
                int oa = srw(qa, 0) * swI, ob = srw(qb, 0) * swI;
                float2 ga0 = f2(pGa[oa]), ga1 = f2(pGa[oa + 1]), gb0 = f2(pGb[ob]), gb1 = f2(pGb[ob + 1]);
                fx2 a0 = pk(f1(pIa[oa]), f1(pIb[ob])), a1 = pk(f1(pIa[oa + 1]), f1(pIb[ob + 1]));
                fx2 hI = fma2(AX, sub2(a1, a0), a0);
                a0 = pk(ga0.x, gb0.x); a1 = pk(ga1.x, gb1.x);
                fx2 hX = fma2(AX, sub2(a1, a0), a0);
                a0 = pk(ga0.y, gb0.y); a1 = pk(ga1.y, gb1.y);
                fx2 hY = fma2(AX, sub2(a1, a0), a0);
#pragma unroll
                for (int e = 0; e < SEG; ++e) {
                    oa = srw(qa, e + 1) * swI; ob = srw(qb, e + 1) * swI;
                    ga0 = f2(pGa[oa]); ga1 = f2(pGa[oa + 1]); gb0 = f2(pGb[ob]); gb1 = f2(pGb[ob + 1]);
                    a0 = pk(f1(pIa[oa]), f1(pIb[ob])); a1 = pk(f1(pIa[oa + 1]), f1(pIb[ob + 1]));
                    const fx2 hI1 = fma2(AX, sub2(a1, a0), a0);
                    a0 = pk(ga0.x, gb0.x); a1 = pk(ga1.x, gb1.x);
                    const fx2 hX1 = fma2(AX, sub2(a1, a0), a0);
                    a0 = pk(ga0.y, gb0.y); a1 = pk(ga1.y, gb1.y);
                    const fx2 hY1 = fma2(AX, sub2(a1, a0), a0);
                    const int m = pp * SEG + e;
                    fx2 t = fma2(AY, sub2(hI1, hI), hI), tx = fma2(AY, sub2(hX1, hX), hX);
                    fx2 ty = fma2(AY, sub2(hY1, hY), hY);
                    if constexpr (!MASK_END) {
                        // samples past the window's last row weigh 0
                        const fx2 ok = pk(sok(qa, e) ? 1.f : 0.f, sok(qb, e) ? 1.f : 0.f), zero = pk(0.f, 0.f);
                        t = fma2(ok, t, zero); tx = fma2(ok, tx, zero); ty = fma2(ok, ty, zero);
                    }
                    tref(m, 0) = t; tref(m, 1) = tx; tref(m, 2) = ty;
                    sxx = fma2(tx, tx, sxx); sxy = fma2(tx, ty, sxy); syy = fma2(ty, ty, syy);
                    hI = hI1; hX = hX1; hY = hY1;
                }
            }
            gxx = psum(sxx, 0);
            gxy = psum(sxy, 0);
            gyy = psum(syy, 0);
        } else {
    #pragma unroll
            for (int q = 0; q < Q; ++q) {
                const PT *pI = sI + offI + scol[q];
                const PT2 *pG = sG + offI + scol[q];
                int o = srw(q, 0) * swI;
                float hI = lerpf(f1(pI[o]), f1(pI[o + 1]), ax);
                float2 g0 = f2(pG[o]), g1 = f2(pG[o + 1]);
                float hX = lerpf(g0.x, g1.x, ax), hY = lerpf(g0.y, g1.y, ax);
    #pragma unroll
                for (int e = 0; e < SEG; ++e) {
                    const int m = q * SEG + e;
                    o = srw(q, e + 1) * swI;
                    const float hI1 = lerpf(f1(pI[o]), f1(pI[o + 1]), ax);
                    g0 = f2(pG[o]); g1 = f2(pG[o + 1]);
                    const float hX1 = lerpf(g0.x, g1.x, ax), hY1 = lerpf(g0.y, g1.y, ax);
                    const bool ok = sok(q, e);
                    const float t = lerpf(hI, hI1, ay), tx = lerpf(hX, hX1, ay), ty = lerpf(hY, hY1, ay);
                    T[m] = ok ? t : 0.f; TX[m] = ok ? tx : 0.f; TY[m] = ok ? ty : 0.f;
                    gxx += TX[m] * TX[m]; gxy += TX[m] * TY[m]; gyy += TY[m] * TY[m];
                    hI = hI1; hX = hX1; hY = hY1;
                }
            }
        }
        group_sum3<WPF>(gxx, gxy, gyy, red, wig, grp);
        ++tpl;
        const float lam = 0.5f * ((gxx + gyy) - sqrtf((gxx - gyy) * (gxx - gyy) + 4.f * gxy * gxy));
        const float det = gxx * gyy - gxy * gxy;
        if (!(lam >= D.min_eig * (float)N) || !(det > 0.f)) {
            vx = ux; vy = uy;
            return false;
        }
        const float idet = 1.f / det;
        float nx = 0.f, ny = 0.f;
        for (int it = 0; it < D.max_iters; ++it) {
            const float qx = fminf(fmaxf(px + gx + nx, -64.f), (float)wl + 64.f);
            const float qy = fminf(fmaxf(py + gy + ny, -64.f), (float)hl + 64.f);
            const float fqx = floorf(qx), fqy = floorf(qy);
            const float cx = qx - fqx, cy = qy - fqy;
            const int jx = (int)fqx - r, jy = (int)fqy - r;
            int ox = jx - jx0, oy = jy - jy0;
            if (ox < 0 || ox > 2 * LK_MARGIN || oy < 0 || oy > 2 * LK_MARGIN) {   // same for the whole group
                jx0 = jx - LK_MARGIN;
                jy0 = jy - LK_MARGIN;
                jin = jx0 >= 0 && jx0 + pj - 1 <= wl - 1 && jy0 >= 0 && jy0 + pj - 1 <= hl - 1;
                group_sync<WPF>(grp);
                if constexpr (TM) {
                    const unsigned char *maps = static_cast<const unsigned char *>(D.tmap);
                    if (maps && jx0 >= 0 && jx0 + TG::PJ <= wl && jy0 >= 0 && jy0 + TG::PJ <= hl) {
                        const int jxa = jx0 & ~(TG::A - 1);
                        offJ = jx0 - jxa;
                        if (tig == 0) {
                            fence_proxy_async();
                            mbar_expect_tx(mb, TG::TX_J);
                            tma_load_2d(sJ, maps + (size_t)((sb * STAB_MAXL + l) * 3 + 2) * 128, jxa, jy0, mb);
                        }
                        if (!mbar_wait(mb, ph)) set_err(D.st, STAB_ERR_TIMEOUT);
                        ph ^= 1u;
                    } else {
                        offJ = stage_k<PT, NT, TG::PJ, TG::BWJ>(Jb, p, wl, hl, jx0, jy0, sJ, tig);
                    }
                } else if constexpr (RC > 0) {
                    constexpr int PJc = 2 * RC + 2 + 2 * LK_MARGIN, SWJ = lk_sw(PJc);
                    offJ = stage_k<PT, NT, PJc, SWJ>(Jb, p, wl, hl, jx0, jy0, sJ, tig);
                } else {
                    offJ = stage<PT, NT>(Jb, p, wl, hl, jx0, jy0, pj, swJ, jin, sJ, tig);
                }
                cpa_wait_all();
                group_sync<WPF>(grp);
                ox = LK_MARGIN;
                oy = LK_MARGIN;
            }
            const PT *sJo = sJ + oy * swJ + ox + offJ;
            float bxs = 0.f, bys = 0.f, unused = 0.f;
            if constexpr (PAIR) {
                const fx2 CX = pk(cx, cx), CY = pk(cy, cy);
                fx2 ax2 = pk(0.f, 0.f), ay2 = ax2;
#pragma unroll
                for (int pp = 0; pp < Q / 2; ++pp) {
                    const int qa = 2 * pp, qb = 2 * pp + 1;
                    const PT *pJa = sJo + scol[qa], *pJb = sJo + scol[qb];
                    int oa = srw(qa, 0) * swJ, ob = srw(qb, 0) * swJ;
                    fx2 a0 = pk(f1(pJa[oa]), f1(pJb[ob])), a1 = pk(f1(pJa[oa + 1]), f1(pJb[ob + 1]));
                    fx2 h = fma2(CX, sub2(a1, a0), a0);
#pragma unroll
                    for (int e = 0; e < SEG; ++e) {
                        oa = srw(qa, e + 1) * swJ; ob = srw(qb, e + 1) * swJ;
                        a0 = pk(f1(pJa[oa]), f1(pJb[ob])); a1 = pk(f1(pJa[oa + 1]), f1(pJb[ob + 1]));
                        const fx2 h1 = fma2(CX, sub2(a1, a0), a0);
                        const int m = pp * SEG + e;
                        const fx2 err = sub2(tref(m, 0), fma2(CY, sub2(h1, h), h));   // outside the window Tx = Ty = 0
                        ax2 = fma2(err, tref(m, 1), ax2);
                        ay2 = fma2(err, tref(m, 2), ay2);
                        h = h1;
                    }
                }
                bxs = psum(ax2, 0);
                bys = psum(ay2, 0);
            } else {
    #pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const PT *pJ = sJo + scol[q];
                    int o = srw(q, 0) * swJ;
                    float h = lerpf(f1(pJ[o]), f1(pJ[o + 1]), cx);
    #pragma unroll
                    for (int e = 0; e < SEG; ++e) {
                        const int m = q * SEG + e;
                        o = srw(q, e + 1) * swJ;
                        const float h1 = lerpf(f1(pJ[o]), f1(pJ[o + 1]), cx);
                        const float err = T[m] - lerpf(h, h1, cy);       // samples outside the window have TX = TY = 0
                        bxs += err * TX[m];
                        bys += err * TY[m];
                        h = h1;
                    }
                }
            }
            if (WPF == 1) { bxs = wsum(bxs); bys = wsum(bys); }
            else group_sum3<WPF>(bxs, bys, unused, red, wig, grp);
            const float ex = (gyy * bxs - gxy * bys) * idet;
            const float ey = (gxx * bys - gxy * bxs) * idet;
            nx += ex; ny += ey;
            ++iters;
            if (ex * ex + ey * ey < D.eps2) break;
        }
        if (l > 0) { gx = 2.f * (gx + nx); gy = 2.f * (gy + ny); }
        else { dx = gx + nx; dy = gy + ny; }
    }
    vx = ux + dx; vy = uy + dy;
    return vx >= 0.f && vx <= (float)(D.w - 1) && vy >= 0.f && vy <= (float)(D.h - 1);
}

// Shared memory per feature group, in bytes, for plane element size es
// (4: FP32, 2: FP16): the template's I and (Ix, Iy) patches ((2r+2) rows of
// stride lk_sw(2r+2)), the next frame's patch ((2r+2+2 margin) rows of stride
// lk_sw(2r+2+2 margin)) and 8 reduction floats; each region 16-byte aligned.
__host__ __device__ constexpr int lk_al16(int b) { return (b + 15) & ~15; }
__host__ __device__ constexpr int lk_bytes_I(int r, int es) { return lk_al16((2 * r + 2) * lk_sw(2 * r + 2) * es); }
__host__ __device__ constexpr int lk_bytes_J(int r, int es)
{
    return lk_al16((2 * r + 2 + 2 * LK_MARGIN) * lk_sw(2 * r + 2 + 2 * LK_MARGIN) * es);
}
// The shared template of a TS group: 3 NS / 2 packed pairs per thread, 32 threads.
__host__ __device__ constexpr int lk_bytes_T(int ns) { return 3 * (ns / 2) * 32 * 8; }
__host__ __device__ constexpr int lk_group_bytes(int r, int es, int tbytes = 0)
{
    return 3 * lk_bytes_I(r, es) + lk_bytes_J(r, es) + 32 + tbytes;
}

template <typename PT, int NS, int RC, int WPF, int MINB, bool TS, bool TM>
__global__ void __launch_bounds__(128, MINB) k_lk(const StreamDev *__restrict__ S, WorkList wl, LkIO io, int rmax)
{
    typedef typename Plane2<PT>::type PT2;
    extern __shared__ __align__(128) unsigned char lk_smem[];
    constexpr int NT = 32 * WPF, ES = (int)sizeof(PT), TB = TS ? lk_bytes_T(NS) : 0;
    const int grp = threadIdx.x / NT, tig = threadIdx.x - grp * NT;
    PT *sI;
    PT2 *sG;
    PT *sJ;
    float *red;
    fx2 *sT = nullptr;
    unsigned long long *mb = nullptr;
    unsigned ph = 0;
    if constexpr (TM) {   // 128-byte aligned boxes (LkTma)
        unsigned char *base = lk_smem + grp * LkTma<PT>::GROUP;
        sI = reinterpret_cast<PT *>(base);
        sG = reinterpret_cast<PT2 *>(base + LkTma<PT>::OFF_G);
        sJ = reinterpret_cast<PT *>(base + LkTma<PT>::OFF_J);
        red = reinterpret_cast<float *>(base + LkTma<PT>::OFF_RED);
        mb = reinterpret_cast<unsigned long long *>(base + LkTma<PT>::OFF_RED + 64);
        if (tig == 0) mbar_init(mb);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        fence_proxy_async();
        group_sync<WPF>(grp);
    } else {
        unsigned char *base = lk_smem + grp * lk_group_bytes(rmax, ES, TB);
        // regions sized for rmax; a stream with a smaller radius uses a prefix
        const int bI = lk_bytes_I(rmax, ES);
        sI = reinterpret_cast<PT *>(base);
        sG = reinterpret_cast<PT2 *>(base + bI);
        sJ = reinterpret_cast<PT *>(base + 3 * bI);
        red = reinterpret_cast<float *>(base + 3 * bI + lk_bytes_J(rmax, ES));
        sT = reinterpret_cast<fx2 *>(base + 3 * bI + lk_bytes_J(rmax, ES) + 32);
    }
    const int ngroups = (gridDim.x * blockDim.x) / NT;
    // The group's next item: a fixed stride, or with a ticket list the ticket
    // thread 0 of the group drew (tk), broadcast to the group.
    int tk = 0;
    auto bcast = [&](int v) {
        if (WPF == 1) return __shfl_sync(0xffffffffu, v, 0);
        group_sync<WPF>(grp);
        if (tig == 0) reinterpret_cast<int *>(red)[7] = v;
        group_sync<WPF>(grp);
        v = reinterpret_cast<const int *>(red)[7];
        group_sync<WPF>(grp);
        return v;
    };
    int first = (blockIdx.x * blockDim.x + threadIdx.x) / NT;
    if (wl.ctr) first = bcast(tig == 0 ? (int)atomicAdd(wl.ctr, 1u) : 0);
    for (int item = first; item < wl.total; item = wl.ctr ? bcast(tk) : item + ngroups) {
        if (wl.ctr && tig == 0) tk = (int)atomicAdd(wl.ctr, 1u);   // drawn now, used after this item
        const int s = wl_stream(wl, item);
        const StreamDev &D = S[s];
        StreamState *st = D.st;
        const int f = item - __ldg(&wl.prefix[s]);
        int n, sp, sn;
        const float2 *pts;
        if (io.pts) { n = io.n; pts = io.pts; sp = io.slot_prev; sn = io.slot_next; }
        else {
            const long long tb = st->t - D.lag;   // frames tb-1 -> tb
            if (tb < 1) continue;
            n = st->n_feat; pts = D.feat; sp = stab_pslot(tb - 1); sn = stab_pslot(tb);
        }
        if (f >= n) continue;
        const float2 u = pts[f];
        int iters = 0, tpl = 0;
        float vx, vy, bx = u.x, by = u.y;
        const bool ok1 = lk_track<PT, NS, RC, WPF, TS, TM>(D, sp, sn, u.x, u.y, vx, vy, iters, tpl, sI, sG, sJ,
                                                           red, sT, mb, ph, tig, grp);
        bool ok2 = false;
        if (ok1) ok2 = lk_track<PT, NS, RC, WPF, TS, TM>(D, sn, sp, vx, vy, bx, by, iters, tpl, sI, sG, sJ, red, sT,
                                                         mb, ph, tig, grp);
        if (!ok1) { bx = u.x; by = u.y; }
        const float ex = bx - u.x, ey = by - u.y;
        const float e2 = ex * ex + ey * ey;
        if (tig == 0) {
            float2 *fwd = io.fwd ? io.fwd : D.fwd;
            float2 *back = io.back ? io.back : D.back;
            float *fb = io.fb ? io.fb : D.fb;
            uint8_t *stt = io.status ? io.status : D.status;
            uint8_t *stf = io.status_fwd ? io.status_fwd : D.status_fwd;
            fwd[f] = make_float2(vx, vy);
            back[f] = make_float2(bx, by);
            fb[f] = ok2 ? sqrtf(e2) : -1.f;
            stt[f] = (uint8_t)(ok1 && ok2 && e2 <= D.fb2);
            stf[f] = (uint8_t)ok1;
            atomicAdd((unsigned long long *)&st->iters, (unsigned long long)iters);
            atomicAdd((unsigned long long *)&st->tpl, (unsigned long long)tpl);
        }
    }
    // every group has drawn a ticket past the end; the last to finish resets the list
    if (wl.ctr && tig == 0 && atomicAdd(wl.ctr + 1, 1u) == (unsigned)(ngroups - 1)) {
        atomicExch(wl.ctr, 0u);
        atomicExch(wl.ctr + 1, 0u);
    }
}

// ---------------------------------------------------------------------------
// Two features per warp for the 21 x 21 window: each half-warp (16 lanes)
// tracks its own feature with its own patches, 28 samples per lane (four
// column segments of 7 rows, run as two pairs in packed f32x2 arithmetic).
// The per-level and per-iteration control (staging, the 2 x 2 solve, the
// convergence test, the loop bookkeeping) is one instruction stream for both
// features, and each lane carries twice the independent arithmetic between
// two reductions (four butterfly steps over the half-warp instead of five).
// The two halves run the same loops with per-half flags: a half whose
// feature is lost, converged or absent idles (its shared memory holds finite
// values, its results are discarded) until the other finishes.

// Sum over the 16 lanes of a half-warp (xor butterfly: the same bits in every lane).
__device__ __forceinline__ float hsum16(float v)
{
#pragma unroll
    for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename PT>
__device__ __noinline__ bool lk_track2(const StreamDev &D, int sa, int sb, bool act, float ux, float uy, float &vx,
                                       float &vy, int &iters, int &tpl, PT *sI, typename Plane2<PT>::type *sG,
                                       PT *sJ, int hl)
{
    typedef typename Plane2<PT>::type PT2;
    constexpr int NT = 16, SEG = 7, Q = 4, ww = 21, pw = ww + 1, N = ww * ww, pj = pw + 2 * LK_MARGIN;
    constexpr int swI = lk_sw(pw), swJ = lk_sw(pj);
    // segments hl + 16 q (q = 0 .. 3): column (hl + 16 q) % 21, rows 7 ((hl + 16 q) / 21) .. + 6; the 64th
    // (lane 15, q = 3) lies past the window and reads rows 0 .. 7 of column 0, dropped from every sum
    int scol[Q], srow[Q];
    bool sv[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int sgi = hl + NT * q;
        sv[q] = sgi < ww * 3;
        scol[q] = sv[q] ? sgi % ww : 0;
        srow[q] = sv[q] ? (sgi / ww) * SEG : 0;
    }
    auto psum = [&](fx2 v, int pp) {
        float u0, u1;
        upk(v, u0, u1);
        return (sv[2 * pp] ? u0 : 0.f) + (sv[2 * pp + 1] ? u1 : 0.f);
    };
    float gx = 0.f, gy = 0.f, dx = 0.f, dy = 0.f;
    fx2 TT[2 * SEG], TTX[2 * SEG], TTY[2 * SEG];
    bool ok = act;
    const int L = act ? D.L : 0, Lw = max(L, __shfl_xor_sync(0xffffffffu, L, 16));
    const int maxit = act ? D.max_iters : 0, maxw = max(maxit, __shfl_xor_sync(0xffffffffu, maxit, 16));
    for (int l = Lw - 1; l >= 0; --l) {
        const bool on = ok && l < L;   // this half works at level l
        const int lc = on ? l : 0;
        const PT *Ia = reinterpret_cast<const PT *>(D.pI[sa][lc]);
        const PT2 *Ga = reinterpret_cast<const PT2 *>(D.pG[sa][lc]);
        const PT *Jb = reinterpret_cast<const PT *>(D.pI[sb][lc]);
        const int wl = D.lw[lc], hlv = D.lh[lc], p = D.lp[lc];
        const float sc = __int_as_float((127 - lc) << 23);   // 2^-l
        const float px = ux * sc, py = uy * sc;
        const float bx = fminf(fmaxf(px, -64.f), (float)wl + 64.f);
        const float by = fminf(fmaxf(py, -64.f), (float)hlv + 64.f);
        const float fx = floorf(bx), fy = floorf(by);
        const float ax = bx - fx, ay = by - fy;
        const int ix = (int)fx - 10, iy = (int)fy - 10;
        int jx0 = (int)floorf(fminf(fmaxf(px + gx, -64.f), (float)wl + 64.f)) - 10 - LK_MARGIN;
        int jy0 = (int)floorf(fminf(fmaxf(py + gy, -64.f), (float)hlv + 64.f)) - 10 - LK_MARGIN;
        __syncwarp();
        int offI = 0, offJ = 0;
        if (on) {
            offI = stage_k<PT, NT, pw, swI>(Ia, p, wl, hlv, ix, iy, sI, hl);
            stage_k<PT2, NT, pw, swI>(Ga, p, wl, hlv, ix, iy, sG, hl);
            offJ = stage_k<PT, NT, pj, swJ>(Jb, p, wl, hlv, jx0, jy0, sJ, hl);
        }
        cpa_wait_all();
        __syncwarp();
        // ---- template T, Tx, Ty and G over the window
        const fx2 AX = pk(ax, ax), AY = pk(ay, ay);
        fx2 sxx[2], sxy[2], syy[2];
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
            const int qa = 2 * pp, qb = 2 * pp + 1;
            sxx[pp] = pk(0.f, 0.f); sxy[pp] = sxx[pp]; syy[pp] = sxx[pp];
            const PT *pIa = sI + offI + scol[qa] + srow[qa] * swI, *pIb = sI + offI + scol[qb] + srow[qb] * swI;
            const PT2 *pGa = sG + offI + scol[qa] + srow[qa] * swI, *pGb = sG + offI + scol[qb] + srow[qb] * swI;
            float2 ga0 = f2(pGa[0]), ga1 = f2(pGa[1]), gb0 = f2(pGb[0]), gb1 = f2(pGb[1]);
            fx2 a0 = pk(f1(pIa[0]), f1(pIb[0])), a1 = pk(f1(pIa[1]), f1(pIb[1]));
            fx2 hI = fma2(AX, sub2(a1, a0), a0);
            a0 = pk(ga0.x, gb0.x); a1 = pk(ga1.x, gb1.x);
            fx2 hX = fma2(AX, sub2(a1, a0), a0);
            a0 = pk(ga0.y, gb0.y); a1 = pk(ga1.y, gb1.y);
            fx2 hY = fma2(AX, sub2(a1, a0), a0);
#pragma unroll
            for (int e = 0; e < SEG; ++e) {
                const int o = (e + 1) * swI;
                ga0 = f2(pGa[o]); ga1 = f2(pGa[o + 1]); gb0 = f2(pGb[o]); gb1 = f2(pGb[o + 1]);
                a0 = pk(f1(pIa[o]), f1(pIb[o])); a1 = pk(f1(pIa[o + 1]), f1(pIb[o + 1]));
                const fx2 hI1 = fma2(AX, sub2(a1, a0), a0);
                a0 = pk(ga0.x, gb0.x); a1 = pk(ga1.x, gb1.x);
                const fx2 hX1 = fma2(AX, sub2(a1, a0), a0);
                a0 = pk(ga0.y, gb0.y); a1 = pk(ga1.y, gb1.y);
                const fx2 hY1 = fma2(AX, sub2(a1, a0), a0);
                const int m = pp * SEG + e;
                TT[m] = fma2(AY, sub2(hI1, hI), hI);
                TTX[m] = fma2(AY, sub2(hX1, hX), hX);
                TTY[m] = fma2(AY, sub2(hY1, hY), hY);
                sxx[pp] = fma2(TTX[m], TTX[m], sxx[pp]);
                sxy[pp] = fma2(TTX[m], TTY[m], sxy[pp]);
                syy[pp] = fma2(TTY[m], TTY[m], syy[pp]);
                hI = hI1; hX = hX1; hY = hY1;
            }
        }
        const float gxx = hsum16(psum(sxx[0], 0) + psum(sxx[1], 1));
        const float gxy = hsum16(psum(sxy[0], 0) + psum(sxy[1], 1));
        const float gyy = hsum16(psum(syy[0], 0) + psum(syy[1], 1));
        if (on) ++tpl;
        const float lam = 0.5f * ((gxx + gyy) - sqrtf((gxx - gyy) * (gxx - gyy) + 4.f * gxy * gxy));
        const float det = gxx * gyy - gxy * gxy;
        if (on && (!(lam >= D.min_eig * (float)N) || !(det > 0.f))) ok = false;
        const float idet = 1.f / det;
        // ---- iterations
        bool run = on && ok;
        float nx = 0.f, ny = 0.f;
        for (int it = 0; it < maxw; ++it) {
            if (!__any_sync(0xffffffffu, run)) break;
            const float qx = fminf(fmaxf(px + gx + nx, -64.f), (float)wl + 64.f);
            const float qy = fminf(fmaxf(py + gy + ny, -64.f), (float)hlv + 64.f);
            const float fqx = floorf(qx), fqy = floorf(qy);
            const float cx = qx - fqx, cy = qy - fqy;
            const int jx = (int)fqx - 10, jy = (int)fqy - 10;
            int ox = jx - jx0, oy = jy - jy0;
            const bool need = run && (ox < 0 || ox > 2 * LK_MARGIN || oy < 0 || oy > 2 * LK_MARGIN);
            if (__any_sync(0xffffffffu, need)) {
                __syncwarp();
                if (need) {
                    jx0 = jx - LK_MARGIN;
                    jy0 = jy - LK_MARGIN;
                    offJ = stage_k<PT, NT, pj, swJ>(Jb, p, wl, hlv, jx0, jy0, sJ, hl);
                }
                cpa_wait_all();
                __syncwarp();
                if (need) { ox = LK_MARGIN; oy = LK_MARGIN; }
            }
            // a half that is not running may hold any offsets: keep its reads inside its patch
            if (!run) { ox = 0; oy = 0; }
            const PT *sJo = sJ + oy * swJ + ox + offJ;
            const fx2 CX = pk(cx, cx), CY = pk(cy, cy);
            float bxs = 0.f, bys = 0.f;
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const int qa = 2 * pp, qb = 2 * pp + 1;
                const PT *pJa = sJo + scol[qa] + srow[qa] * swJ, *pJb = sJo + scol[qb] + srow[qb] * swJ;
                fx2 a0 = pk(f1(pJa[0]), f1(pJb[0])), a1 = pk(f1(pJa[1]), f1(pJb[1]));
                fx2 h = fma2(CX, sub2(a1, a0), a0);
                fx2 ax2 = pk(0.f, 0.f), ay2 = ax2;
#pragma unroll
                for (int e = 0; e < SEG; ++e) {
                    const int o = (e + 1) * swJ;
                    a0 = pk(f1(pJa[o]), f1(pJb[o])); a1 = pk(f1(pJa[o + 1]), f1(pJb[o + 1]));
                    const fx2 h1 = fma2(CX, sub2(a1, a0), a0);
                    const int m = pp * SEG + e;
                    const fx2 err = sub2(TT[m], fma2(CY, sub2(h1, h), h));
                    ax2 = fma2(err, TTX[m], ax2);
                    ay2 = fma2(err, TTY[m], ay2);
                    h = h1;
                }
                bxs += psum(ax2, pp);
                bys += psum(ay2, pp);
            }
            bxs = hsum16(bxs);
            bys = hsum16(bys);
            if (run) {
                const float ex = (gyy * bxs - gxy * bys) * idet;
                const float ey = (gxx * bys - gxy * bxs) * idet;
                nx += ex; ny += ey;
                ++iters;
                if (ex * ex + ey * ey < D.eps2 || it + 1 >= maxit) run = false;
            }
        }
        if (on && ok) {
            if (l > 0) { gx = 2.f * (gx + nx); gy = 2.f * (gy + ny); }
            else { dx = gx + nx; dy = gy + ny; }
        }
    }
    if (!ok) { vx = ux; vy = uy; return false; }
    vx = ux + dx; vy = uy + dy;
    return vx >= 0.f && vx <= (float)(D.w - 1) && vy >= 0.f && vy <= (float)(D.h - 1);
}

template <typename PT, int MINB>
__global__ void __launch_bounds__(128, MINB) k_lk2(const StreamDev *__restrict__ S, WorkList wl, LkIO io)
{
    typedef typename Plane2<PT>::type PT2;
    extern __shared__ __align__(128) unsigned char lk_smem[];
    constexpr int ES = (int)sizeof(PT);
    const int grp = threadIdx.x >> 4, hl = threadIdx.x & 15;
    unsigned char *base = lk_smem + grp * lk_group_bytes(10, ES);
    const int bI = lk_bytes_I(10, ES);
    PT *sI = reinterpret_cast<PT *>(base);
    PT2 *sG = reinterpret_cast<PT2 *>(base + bI);
    PT *sJ = reinterpret_cast<PT *>(base + 3 * bI);
    const int ngroups = (gridDim.x * blockDim.x) >> 4;
    auto bcast = [](int v) { return __shfl_sync(0xffffffffu, v, 0, 16); };   // from lane 0 of each half
    int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 4, tk = 0;
    if (wl.ctr) item = bcast(hl == 0 ? (int)atomicAdd(wl.ctr, 1u) : 0);
    while (__any_sync(0xffffffffu, item < wl.total)) {
        const bool have = item < wl.total;
        if (wl.ctr && hl == 0 && have) tk = (int)atomicAdd(wl.ctr, 1u);   // drawn now, used after this item
        const int s = have ? wl_stream(wl, item) : 0;
        const StreamDev &D = S[s];
        StreamState *st = D.st;
        const int f = have ? item - __ldg(&wl.prefix[s]) : 0;
        int n = 0, sp = 0, sn = 1;
        const float2 *pts = D.feat;
        if (io.pts) { n = io.n; pts = io.pts; sp = io.slot_prev; sn = io.slot_next; }
        else if (have) {
            const long long tb = st->t - D.lag;   // frames tb-1 -> tb
            if (tb >= 1) { n = st->n_feat; sp = stab_pslot(tb - 1); sn = stab_pslot(tb); }
        }
        const bool valid = have && f < n;
        const float2 u = valid ? pts[f] : make_float2(0.f, 0.f);
        int iters = 0, tpl = 0;
        float vx, vy, bx = u.x, by = u.y;
        const bool ok1 = lk_track2<PT>(D, sp, sn, valid, u.x, u.y, vx, vy, iters, tpl, sI, sG, sJ, hl);
        const bool ok2 = lk_track2<PT>(D, sn, sp, valid && ok1, vx, vy, bx, by, iters, tpl, sI, sG, sJ, hl) &&
                         valid && ok1;
        if (!ok1) { bx = u.x; by = u.y; }
        const float ex = bx - u.x, ey = by - u.y;
        const float e2 = ex * ex + ey * ey;
        if (valid && hl == 0) {
            float2 *fwd = io.fwd ? io.fwd : D.fwd;
            float2 *back = io.back ? io.back : D.back;
            float *fb = io.fb ? io.fb : D.fb;
            uint8_t *stt = io.status ? io.status : D.status;
            uint8_t *stf = io.status_fwd ? io.status_fwd : D.status_fwd;
            fwd[f] = make_float2(vx, vy);
            back[f] = make_float2(bx, by);
            fb[f] = ok2 ? sqrtf(e2) : -1.f;
            stt[f] = (uint8_t)(ok1 && ok2 && e2 <= D.fb2);
            stf[f] = (uint8_t)ok1;
            atomicAdd((unsigned long long *)&st->iters, (unsigned long long)iters);
            atomicAdd((unsigned long long *)&st->tpl, (unsigned long long)tpl);
        }
        if (have) item = wl.ctr ? tk : item + ngroups;
        item = wl.ctr ? bcast(item) : item;
    }
    // every half has drawn a ticket past the end; the last to finish resets the list
    if (wl.ctr && hl == 0 && atomicAdd(wl.ctr + 1, 1u) == (unsigned)(ngroups - 1)) {
        atomicExch(wl.ctr, 0u);
        atomicExch(wl.ctr + 1, 0u);
    }
}

template <typename PT, int MINB>
struct Lk2Kernel {
    static int smem() { return 8 * lk_group_bytes(10, (int)sizeof(PT)); }
    static int occ()
    {
        static DevCache c;
        return c.get([] {
            int v = 0;
            cudaFuncSetAttribute(k_lk2<PT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem());
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_lk2<PT, MINB>, 128, smem()) != cudaSuccess || v < 1)
                v = 1;
            return v;
        });
    }
    static void run(const Launch &L, const StreamDev *S, WorkList wl, LkIO io)
    {
        const int blocks = (wl.total + 7) / 8;
        k_lk2<PT, MINB><<<grid_for(L, blocks, occ()), 128, smem(), L.stream>>>(S, wl, io);
    }
};

template <typename PT, int NS, int RC, int WPF, int MINB, bool TS = false, bool TM = false>
struct LkKernel {
    static int smem(int rmax)
    {
        if (TM) return (128 / (32 * WPF)) * LkTma<PT>::GROUP;
        return (128 / (32 * WPF)) * lk_group_bytes(rmax, (int)sizeof(PT), TS ? lk_bytes_T(NS) : 0);
    }
    // sets the kernel's shared-memory attribute and queries its occupancy, once
    // per device and radius
    static int occ(int rmax)
    {
        static DevCache c[STAB_MAXR + 1];
        return c[rmax].get([rmax] {
            int v = 0;
            cudaFuncSetAttribute(k_lk<PT, NS, RC, WPF, MINB, TS, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem(rmax));
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_lk<PT, NS, RC, WPF, MINB, TS, TM>, 128, smem(rmax)) !=
                    cudaSuccess ||
                v < 1)
                v = 1;
            return v;
        });
    }
    static void run(const Launch &L, const StreamDev *S, WorkList wl, LkIO io, int rmax)
    {
        const int groups_per_block = 128 / (32 * WPF);
        const int blocks = (wl.total + groups_per_block - 1) / groups_per_block;
        k_lk<PT, NS, RC, WPF, MINB, TS, TM><<<grid_for(L, blocks, occ(rmax)), 128, smem(rmax), L.stream>>>(S, wl, io,
                                                                                                      rmax);
    }
};

// Variants for the 21 x 21 window (radius known at compile time):
//   0: one warp per feature, <= 128 registers (4 blocks / SM)
//   1: one warp per feature, <= 168 registers (3 blocks / SM)
//   2: two warps per feature, <= 80 registers (6 blocks / SM)
//   3: two warps per feature, <= 128 registers (4 blocks / SM)
//   4: one warp per feature, template in shared memory, <= 96 registers
//      (5 blocks / SM with FP16 planes: 10.5 KB of shared memory per warp)
//   5, 6: two features per warp (a half-warp each), <= 255 / 168 registers
//      (2 / 3 blocks of 4 warps per SM)
//   7, 8: as 0 / 1, patches inside their level staged by tensor copies
// Other radii use the runtime-radius build of variant 0.
// rcode: the window radius shared by every stream, or minus the largest
// radius when streams differ (then the runtime-radius build, sized for it).
template <typename PT>
void run_variant(int v, const Launch &L, const StreamDev *S, WorkList wl, LkIO io, int rcode)
{
    if (rcode == 10) {
        switch (v) {
        case 1: LkKernel<PT, 14, 10, 1, 3>::run(L, S, wl, io, 10); return;
        case 2: LkKernel<PT, 7, 10, 2, 6>::run(L, S, wl, io, 10); return;
        case 3: LkKernel<PT, 7, 10, 2, 4>::run(L, S, wl, io, 10); return;
        case 4: LkKernel<PT, 14, 10, 1, 5, true>::run(L, S, wl, io, 10); return;
        case 5: Lk2Kernel<PT, 2>::run(L, S, wl, io); return;
        case 6: Lk2Kernel<PT, 3>::run(L, S, wl, io); return;
        case 7: LkKernel<PT, 14, 10, 1, 4, false, true>::run(L, S, wl, io, 10); return;
        case 8: LkKernel<PT, 14, 10, 1, 3, false, true>::run(L, S, wl, io, 10); return;
        default: LkKernel<PT, 14, 10, 1, 4>::run(L, S, wl, io, 10); return;
        }
    }
    const int rmax = rcode < 0 ? -rcode : rcode;
    if (rmax <= 10) LkKernel<PT, 14, 0, 1, 4>::run(L, S, wl, io, rmax);
    else LkKernel<PT, 20, 0, 1, 3>::run(L, S, wl, io, rmax);
}

template <typename PT>
void warm_all()
{
    for (int r = 1; r <= STAB_MAXR; ++r) {
        if (r == 10) {
            LkKernel<PT, 14, 10, 1, 4>::occ(r); LkKernel<PT, 14, 10, 1, 3>::occ(r);
            LkKernel<PT, 7, 10, 2, 6>::occ(r); LkKernel<PT, 7, 10, 2, 4>::occ(r);
            LkKernel<PT, 14, 10, 1, 5, true>::occ(r);
            Lk2Kernel<PT, 2>::occ(); Lk2Kernel<PT, 3>::occ();
            LkKernel<PT, 14, 10, 1, 4, false, true>::occ(r); LkKernel<PT, 14, 10, 1, 3, false, true>::occ(r);
            LkKernel<PT, 14, 0, 1, 4>::occ(r);
        } else if (r < 10) {
            LkKernel<PT, 14, 0, 1, 4>::occ(r);
        } else {
            LkKernel<PT, 20, 0, 1, 3>::occ(r);
        }
    }
}

}  // namespace

int lk_variants() { return 9; }

// Tensor maps of one stream's tracker planes: for every pyramid slot and
// level, the template's I box (BWI x 22), its (Ix, Iy) box (BWI x 22) and the
// next frame's I box (BWJ x 26), each over the level's w x h plane with its
// pitch; columns past w read zero (never sampled).
int lk_tensor_maps(const StreamDev &D, int prec, void *host_out)
{
    typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeFn>(f);
    }();
    if (!encode) return -1;
    const int es = prec ? 2 : 4;
    const int bwi = prec ? LkTma<__half>::BWI : LkTma<float>::BWI, bwj = prec ? LkTma<__half>::BWJ : LkTma<float>::BWJ;
    const CUtensorMapDataType ti = prec ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
    const CUtensorMapDataType tg = prec ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64;
    std::vector<CUtensorMap> maps(STAB_PSLOTS * STAB_MAXL * 3);
    std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    const cuuint32_t one[2] = {1, 1};
    for (int s = 0; s < STAB_PSLOTS; ++s)
        for (int l = 0; l < D.L; ++l) {
            const cuuint64_t dim[2] = {(cuuint64_t)D.lw[l], (cuuint64_t)D.lh[l]};
            const cuuint64_t si[1] = {(cuuint64_t)D.lp[l] * es}, sg[1] = {(cuuint64_t)D.lp[l] * 2 * es};
            const cuuint32_t bi[2] = {(cuuint32_t)bwi, 22}, bj[2] = {(cuuint32_t)bwj, 26};
            CUtensorMap *m = &maps[(s * STAB_MAXL + l) * 3];
            if (encode(m, ti, 2, D.pI[s][l], dim, si, bi, one, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
                encode(m + 1, tg, 2, D.pG[s][l], dim, sg, bi, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
                encode(m + 2, ti, 2, D.pI[s][l], dim, si, bj, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return -1;
        }
    std::memcpy(host_out, maps.data(), maps.size() * sizeof(CUtensorMap));
    return 0;
}

void warm_lk()
{
    warm_all<float>();
    warm_all<__half>();
}

void launch_lk(const Launch &L, int prec, int rcode, int variant, const StreamDev *S, WorkList wl, LkIO io)
{
    if (prec) run_variant<__half>(variant, L, S, wl, io, rcode);
    else run_variant<float>(variant, L, S, wl, io, rcode);
}

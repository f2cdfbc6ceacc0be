// k_lk.cu -- pyramidal Lucas-Kanade (Sec. 3.2, Eq. 3-6; coarse-to-fine as in
// Bouguet's pyramidal implementation cited there) with the forward-backward
// check of Sec. 4.1.
//
// One warp tracks one feature.  The (2r+1)^2 window is spread over the 32
// lanes (NS samples per lane).  At each level the template I, Ix, Iy is
// sampled once, bilinearly, with weights shared by every sample (the window
// sits at integer offsets from the point), and kept in registers; each
// iteration samples the next frame at the displaced window, accumulates
// b = sum e [Ix, Iy], and solves the 2x2 system.  The three G sums and the
// two b sums are reduced with xor-butterfly shuffles, which leave the same
// bits in every lane, so the convergence test is warp-uniform.  Arithmetic
// is FP32 for both storage precisions of the planes.
#include "kernels.cuh"

namespace {

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename PT, int NS>
__device__ bool lk_track(const StreamDev &D, int sa, int sb, float ux, float uy, float &vx, float &vy, int &iters,
                         int &tpl)
{
    typedef typename Plane2<PT>::type PT2;
    const int lane = threadIdx.x & 31;
    const int r = D.r, ww = 2 * r + 1, N = ww * ww;
    const int q32 = 32 / ww, r32 = 32 - q32 * ww;
    const int i_l0 = lane % ww, j_l0 = lane / ww;
    float gx = 0.f, gy = 0.f, dx = 0.f, dy = 0.f;
    float T[NS], TX[NS], TY[NS];
    for (int l = D.L - 1; l >= 0; --l) {
        const PT *Ia = reinterpret_cast<const PT *>(D.pI[sa][l]);
        const PT2 *Ga = reinterpret_cast<const PT2 *>(D.pG[sa][l]);
        const PT *Jb = reinterpret_cast<const PT *>(D.pI[sb][l]);
        const int wl = D.lw[l], hl = D.lh[l], p = D.lp[l];
        const float sc = __int_as_float((127 - l) << 23);   // 2^-l
        const float px = ux * sc, py = uy * sc;
        {
            const float bx = fminf(fmaxf(px, -64.f), (float)wl + 64.f);
            const float by = fminf(fmaxf(py, -64.f), (float)hl + 64.f);
            const float fx = floorf(bx), fy = floorf(by);
            const float ax = bx - fx, ay = by - fy;
            const int ix = (int)fx - r, iy = (int)fy - r;
            const float w00 = (1.f - ax) * (1.f - ay), w01 = ax * (1.f - ay);
            const float w10 = (1.f - ax) * ay, w11 = ax * ay;
            const bool inside = ix >= 0 && ix + ww <= wl - 1 && iy >= 0 && iy + ww <= hl - 1;
            float gxx = 0.f, gxy = 0.f, gyy = 0.f;
            int i = i_l0, j = j_l0;
#pragma unroll
            for (int m = 0; m < NS; ++m) {
                const int k = lane + 32 * m;
                T[m] = 0.f; TX[m] = 0.f; TY[m] = 0.f;
                if (k < N) {
                    int xa = ix + i, ya = iy + j, xb = xa + 1, yb = ya + 1;
                    if (!inside) {
                        xa = clampi(xa, 0, wl - 1); xb = clampi(xb, 0, wl - 1);
                        ya = clampi(ya, 0, hl - 1); yb = clampi(yb, 0, hl - 1);
                    }
                    const size_t ra = (size_t)ya * p, rb = (size_t)yb * p;
                    const float t = w00 * ld1(Ia + ra + xa) + w01 * ld1(Ia + ra + xb) + w10 * ld1(Ia + rb + xa) +
                                    w11 * ld1(Ia + rb + xb);
                    const float2 g00 = ld2(Ga + ra + xa), g01 = ld2(Ga + ra + xb);
                    const float2 g10 = ld2(Ga + rb + xa), g11 = ld2(Ga + rb + xb);
                    const float tx = w00 * g00.x + w01 * g01.x + w10 * g10.x + w11 * g11.x;
                    const float ty = w00 * g00.y + w01 * g01.y + w10 * g10.y + w11 * g11.y;
                    T[m] = t; TX[m] = tx; TY[m] = ty;
                    gxx += tx * tx; gxy += tx * ty; gyy += ty * ty;
                }
                i += r32; j += q32;
                if (i >= ww) { i -= ww; ++j; }
            }
            gxx = wsum(gxx); gxy = wsum(gxy); gyy = wsum(gyy);
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
                const float v00 = (1.f - cx) * (1.f - cy), v01 = cx * (1.f - cy);
                const float v10 = (1.f - cx) * cy, v11 = cx * cy;
                const bool jin = jx >= 0 && jx + ww <= wl - 1 && jy >= 0 && jy + ww <= hl - 1;
                float bxs = 0.f, bys = 0.f;
                int i2 = i_l0, j2 = j_l0;
#pragma unroll
                for (int m = 0; m < NS; ++m) {
                    const int k = lane + 32 * m;
                    if (k < N) {
                        int xa = jx + i2, ya = jy + j2, xb = xa + 1, yb = ya + 1;
                        if (!jin) {
                            xa = clampi(xa, 0, wl - 1); xb = clampi(xb, 0, wl - 1);
                            ya = clampi(ya, 0, hl - 1); yb = clampi(yb, 0, hl - 1);
                        }
                        const size_t ra = (size_t)ya * p, rb = (size_t)yb * p;
                        const float jv = v00 * ld1(Jb + ra + xa) + v01 * ld1(Jb + ra + xb) +
                                         v10 * ld1(Jb + rb + xa) + v11 * ld1(Jb + rb + xb);
                        const float e = T[m] - jv;
                        bxs += e * TX[m];
                        bys += e * TY[m];
                    }
                    i2 += r32; j2 += q32;
                    if (i2 >= ww) { i2 -= ww; ++j2; }
                }
                bxs = wsum(bxs); bys = wsum(bys);
                const float ex = (gyy * bxs - gxy * bys) * idet;
                const float ey = (gxx * bys - gxy * bxs) * idet;
                nx += ex; ny += ey;
                ++iters;
                if (ex * ex + ey * ey < D.eps2) break;
            }
            if (l > 0) { gx = 2.f * (gx + nx); gy = 2.f * (gy + ny); }
            else { dx = gx + nx; dy = gy + ny; }
        }
    }
    vx = ux + dx; vy = uy + dy;
    return vx >= 0.f && vx <= (float)(D.w - 1) && vy >= 0.f && vy <= (float)(D.h - 1);
}

template <typename PT, int NS>
__global__ void __launch_bounds__(128) k_lk(const StreamDev *__restrict__ S, WorkList wl, LkIO io)
{
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < wl.total; item += nw) {
        const int s = wl_stream(wl, item);
        const StreamDev &D = S[s];
        StreamState *st = D.st;
        const int f = item - __ldg(&wl.prefix[s]);
        int n, sp;
        const float2 *pts;
        if (io.pts) { n = io.n; pts = io.pts; sp = io.slot_prev; }
        else {
            if (st->t < 1) continue;
            n = st->n_feat; pts = D.feat; sp = (int)((st->t - 1) & 1);
        }
        if (f >= n) continue;
        const float2 u = pts[f];
        int iters = 0, tpl = 0;
        float vx, vy, bx = u.x, by = u.y;
        const bool ok1 = lk_track<PT, NS>(D, sp, sp ^ 1, u.x, u.y, vx, vy, iters, tpl);
        bool ok2 = false;
        if (ok1) ok2 = lk_track<PT, NS>(D, sp ^ 1, sp, vx, vy, bx, by, iters, tpl);
        if (!ok2) { if (!ok1) { bx = u.x; by = u.y; } }
        const float ex = bx - u.x, ey = by - u.y;
        const float e2 = ex * ex + ey * ey;
        if (lane == 0) {
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
}

template <typename PT, int NS>
int occ_lk()
{
    static int v = 0;
    if (!v && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_lk<PT, NS>, 128, 0) != cudaSuccess || v < 1))
        v = 1;
    return v;
}

template <typename PT, int NS>
void run_lk(const Launch &L, const StreamDev *S, WorkList wl, LkIO io)
{
    int blocks = (wl.total + 3) / 4;
    k_lk<PT, NS><<<grid_for(L, blocks, occ_lk<PT, NS>()), 128, 0, L.stream>>>(S, wl, io);
}

}  // namespace

void warm_lk()
{
    occ_lk<float, 14>(); occ_lk<__half, 14>(); occ_lk<float, 20>(); occ_lk<__half, 20>();
}

void launch_lk(const Launch &L, int prec, int r, int wpf, const StreamDev *S, WorkList wl, LkIO io)
{
    (void)wpf;
    if (r <= 10) {
        if (prec) run_lk<__half, 14>(L, S, wl, io);
        else run_lk<float, 14>(L, S, wl, io);
    } else {
        if (prec) run_lk<__half, 20>(L, S, wl, io);
        else run_lk<float, 20>(L, S, wl, io);
    }
}

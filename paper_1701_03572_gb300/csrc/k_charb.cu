// k_charb.cu -- photometric refinement of the similarity of Sec. 4 through
// the warp of Sec. 5.1: Charbonnier loss of the warped current frame against
// the previous frame, its hand-written adjoint, and Gauss-Newton.
//
//   L = sum_{x in Omega} rho(r),  rho(r) = sqrt(r^2 + eps^2),
//   r = I_t(W(x)) - I_prev(x),    W(x) = c + s R(th) (x - c) + t.
//
// k_charb_fwd: one CTA per frame pair; each thread walks a strided share of
// Omega and accumulates 19 sums (loss, dL/dtheta, the 10 upper entries of the
// IRLS normal matrix H = sum J^T J / rho and g = sum J^T r / rho); a fixed-order
// block reduction makes the result deterministic.  With `update` set, thread 0
// solves H d = g (FP64 Cholesky, 4x4) and applies theta -= d in place: one
// launch per Gauss-Newton step, no scratch memory.
// k_charb_bwd_img: dL/dI_t by gathering, for every pixel q of I_t, the output
// samples whose bilinear footprint contains q (found by mapping q's 2x2 cell
// back through W^-1), in a fixed order; dL/dI_prev = -rho'(r) on Omega.
#include "kernels.cuh"

namespace {

struct Sim {
    float cx, cy, s, c, sn, tx, ty, A, B;
};

// W(x) - x = (s cos th - 1) dx - s sin th dy + tx (and likewise for y), with
// s cos th - 1 = expm1(log s) cos th - 2 sin^2(th / 2) formed from small terms,
// so that the displacement (not the absolute position, ~1e3 px) carries the
// FP32 rounding: the residual r then keeps ~1e-6 absolute accuracy, which the
// Charbonnier slope r / sqrt(r^2 + eps^2) (up to 1 / eps per unit of r) needs.
__device__ __forceinline__ Sim make_sim(const float *th, int w, int h)
{
    Sim m;
    m.cx = 0.5f * (float)(w - 1);
    m.cy = 0.5f * (float)(h - 1);
    m.s = expf(th[3]);
    sincosf(th[2], &m.sn, &m.c);
    const float hs = sinf(0.5f * th[2]);
    m.A = expm1f(th[3]) * m.c - 2.f * hs * hs;
    m.B = m.s * m.sn;
    m.tx = th[0];
    m.ty = th[1];
    return m;
}

// Sample of I_t at W(x, y) (zero outside), the residual against I_prev
// formed from differences of neighbouring values, and the gradient of the
// bilinear interpolant; rx, ry = R (x - c).
struct Samp {
    float r, gx, gy, rx, ry, ax, ay;
    int x0, y0;
};

__device__ __forceinline__ Samp sample(const float *__restrict__ I, float Ipx, int w, int h, const Sim &m, int x,
                                       int y)
{
    Samp o;
    const float dx = (float)x - m.cx, dy = (float)y - m.cy;
    o.rx = m.c * dx - m.sn * dy;
    o.ry = m.sn * dx + m.c * dy;
    const float ddx = fmaf(m.A, dx, fmaf(-m.B, dy, m.tx));
    const float ddy = fmaf(m.B, dx, fmaf(m.A, dy, m.ty));
    const float fx = floorf(ddx), fy = floorf(ddy);
    o.ax = ddx - fx;
    o.ay = ddy - fy;
    o.x0 = x + (int)fminf(fmaxf(fx, -(float)w - 2.f), (float)w + 2.f);
    o.y0 = y + (int)fminf(fmaxf(fy, -(float)h - 2.f), (float)h + 2.f);
    const int x0 = o.x0, y0 = o.y0;
    auto tap = [&](int xx, int yy) -> float {
        return (xx >= 0 && xx < w && yy >= 0 && yy < h) ? __ldg(I + (size_t)yy * w + xx) : 0.f;
    };
    const float p00 = tap(x0, y0), p01 = tap(x0 + 1, y0), p10 = tap(x0, y0 + 1), p11 = tap(x0 + 1, y0 + 1);
    const float d1 = p01 - p00, d2 = p10 - p00, d3 = (p11 - p10) - d1;
    o.r = fmaf(o.ax * o.ay, d3, fmaf(o.ay, d2, fmaf(o.ax, d1, p00 - Ipx)));
    o.gx = fmaf(o.ay, d3, d1);
    o.gy = fmaf(o.ax, d3, d2);
    return o;
}

constexpr int NSUM = 19;   // loss, dtheta[4], H upper[10], g[4]

__global__ void __launch_bounds__(1024) k_charb_fwd(const float *__restrict__ It, const float *__restrict__ Ip, int w,
                                                    int h, float *theta, int margin, float eps, float *loss,
                                                    float *dtheta, float *gn, int update)
{
    __shared__ float sred[32][NSUM];
    __shared__ float sfin[NSUM];
    const int p = blockIdx.x;
    const size_t plane = (size_t)w * h;
    const float *I = It + p * plane, *J0 = Ip + p * plane;
    float th[4];
    for (int k = 0; k < 4; ++k) th[k] = theta[4 * p + k];
    const Sim m = make_sim(th, w, h);
    const float e2 = eps * eps;
    float acc[NSUM];
#pragma unroll
    for (int k = 0; k < NSUM; ++k) acc[k] = 0.f;
    const int ow = w - 2 * margin, oh = h - 2 * margin;
    const int npx = ow > 0 && oh > 0 ? ow * oh : 0;
    for (int i = threadIdx.x; i < npx; i += blockDim.x) {
        const int y = margin + i / ow, x = margin + i % ow;
        const Samp S = sample(I, __ldg(J0 + (size_t)y * w + x), w, h, m, x, y);
        const float r = S.r;
        const float rho = sqrtf(r * r + e2);
        const float irho = 1.f / rho;
        const float psi = r * irho;
        const float Jv[4] = {S.gx, S.gy, m.s * (-S.ry * S.gx + S.rx * S.gy), m.s * (S.rx * S.gx + S.ry * S.gy)};
        acc[0] += rho;
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[1 + a] += psi * Jv[a];
        int k = 5;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a; b < 4; ++b) acc[k++] += irho * Jv[a] * Jv[b];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[15 + a] += irho * Jv[a] * r;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NSUM; ++k) {
        float v = acc[k];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sred[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NSUM) {
        float a = 0.f;
        for (int i = 0; i < nw; ++i) a += sred[i][threadIdx.x];
        sfin[threadIdx.x] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (loss) loss[p] = sfin[0];
        if (dtheta)
            for (int a = 0; a < 4; ++a) dtheta[4 * p + a] = sfin[1 + a];
        if (gn)
            for (int k = 0; k < 14; ++k) gn[14 * p + k] = sfin[5 + k];
        if (update) {
            double Hm[4][4], g[4], L[4][4] = {{0}};
            int k = 5;
            for (int a = 0; a < 4; ++a)
                for (int b = a; b < 4; ++b) Hm[a][b] = Hm[b][a] = sfin[k++];
            for (int a = 0; a < 4; ++a) g[a] = sfin[15 + a];
            bool ok = true;
            for (int i = 0; i < 4 && ok; ++i)
                for (int j = 0; j <= i; ++j) {
                    double s = Hm[i][j];
                    for (int q = 0; q < j; ++q) s -= L[i][q] * L[j][q];
                    if (i == j) {
                        if (!(s > 0.0)) { ok = false; break; }
                        L[i][i] = sqrt(s);
                    } else {
                        L[i][j] = s / L[j][j];
                    }
                }
            if (ok) {
                double z[4], d[4];
                for (int i = 0; i < 4; ++i) {
                    double s = g[i];
                    for (int q = 0; q < i; ++q) s -= L[i][q] * z[q];
                    z[i] = s / L[i][i];
                }
                for (int i = 3; i >= 0; --i) {
                    double s = z[i];
                    for (int q = i + 1; q < 4; ++q) s -= L[q][i] * d[q];
                    d[i] = s / L[i][i];
                }
                for (int a = 0; a < 4; ++a) theta[4 * p + a] = (float)((double)th[a] - d[a]);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_charb_bwd_img(const float *__restrict__ It, const float *__restrict__ Ip,
                                                       int w, int h, int P, const float *__restrict__ theta, int margin,
                                                       float eps, const float *__restrict__ gout, float *dIt,
                                                       float *dIp)
{
    const size_t plane = (size_t)w * h;
    const size_t total = plane * P;
    const float e2 = eps * eps;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx / plane);
        const int q = (int)(idx - (size_t)p * plane);
        const int qy = q / w, qx = q - qy * w;
        const float *I = It + p * plane, *J0 = Ip + p * plane;
        const float go = gout ? gout[p] : 1.f;
        float th[4];
        for (int k = 0; k < 4; ++k) th[k] = theta[4 * p + k];
        const Sim m = make_sim(th, w, h);
        if (dIp) {
            float v = 0.f;
            if (qx >= margin && qx < w - margin && qy >= margin && qy < h - margin) {
                const Samp S = sample(I, __ldg(J0 + q), w, h, m, qx, qy);
                v = -go * S.r / sqrtf(S.r * S.r + e2);
            }
            dIp[idx] = v;
        }
        if (!dIt) continue;
        // output pixels x whose W(x) lies in (qx-1, qx+1) x (qy-1, qy+1):
        // x = c + R(-th) (W - c - t) / s, bounding box of the cell's corners
        const float is = 1.f / m.s;
        float xmin = 1e30f, xmax = -1e30f, ymin = 1e30f, ymax = -1e30f;
        for (int k = 0; k < 4; ++k) {
            const float Wx = (float)qx + ((k & 1) ? 1.f : -1.f), Wy = (float)qy + ((k & 2) ? 1.f : -1.f);
            const float ux = Wx - m.cx - m.tx, uy = Wy - m.cy - m.ty;
            const float xx = m.cx + is * (m.c * ux + m.sn * uy), yy = m.cy + is * (-m.sn * ux + m.c * uy);
            xmin = fminf(xmin, xx); xmax = fmaxf(xmax, xx);
            ymin = fminf(ymin, yy); ymax = fmaxf(ymax, yy);
        }
        const int x0 = max(margin, (int)floorf(xmin) - 1), x1 = min(w - margin - 1, (int)ceilf(xmax) + 1);
        const int y0 = max(margin, (int)floorf(ymin) - 1), y1 = min(h - margin - 1, (int)ceilf(ymax) + 1);
        float g = 0.f;
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                const Samp S = sample(I, __ldg(J0 + (size_t)y * w + x), w, h, m, x, y);
                const int dxq = qx - S.x0, dyq = qy - S.y0;
                if (dxq < 0 || dxq > 1 || dyq < 0 || dyq > 1) continue;
                const float wgt = (dxq ? S.ax : 1.f - S.ax) * (dyq ? S.ay : 1.f - S.ay);
                g += wgt * S.r / sqrtf(S.r * S.r + e2);
            }
        dIt[idx] = go * g;
    }
}

}  // namespace

void launch_charb_forward(const Launch &L, const float *It, const float *Ip, int w, int h, int P, float *theta,
                          int margin, float eps, float *loss, float *dtheta, float *gn, int update)
{
    k_charb_fwd<<<P, 1024, 0, L.stream>>>(It, Ip, w, h, theta, margin, eps, loss, dtheta, gn, update);
}

void launch_charb_backward_image(const Launch &L, const float *It, const float *Ip, int w, int h, int P,
                                 const float *theta, int margin, float eps, const float *gout, float *dIt, float *dIp)
{
    const long long total = (long long)w * h * P;
    long long g = (total + 255) / 256;
    if (g > 8LL * L.sms * 8) g = 8LL * L.sms * 8;
    k_charb_bwd_img<<<(int)g, 256, 0, L.stream>>>(It, Ip, w, h, P, theta, margin, eps, gout, dIt, dIp);
}

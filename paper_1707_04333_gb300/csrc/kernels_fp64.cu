// Plain-FP64 kernels of the FETD-PIC step (Faraday update + the fused
// gather / push / walk / deposit particle kernel).
//
// This file is compiled with -fmad=false: every multiply and add rounds as
// written, in the order written, so a step from a given state reproduces a
// plain FP64 evaluation of the paper's formulas bit for bit (cells, crossed
// edges, positions, momenta).  Division and square root are IEEE
// correctly-rounded in CUDA and so also reproducible.
#include <cuda_runtime.h>

#include "fetdpic_internal.h"

namespace fetdpic {

// Faraday, Eq. (semi.dis.curl.1): b^{n+1/2} = b^{n-1/2} - dt C e^n, in place,
// fused with the per-triangle field record the particles gather from:
// (s_m e_m) for the three local edges and B_z^n = (b^{n+1/2}+b^{n-1/2})/(2A).
__global__ void k_faraday64(int F, const Geo64 *__restrict__ geo, const Topo *__restrict__ topo,
                            const double *__restrict__ e, double *__restrict__ b, Rec64 *__restrict__ rec)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const Topo t = topo[f];
    double se[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const double v = e[t.ew[m] >> 1];
        se[m] = (t.ew[m] & 1) ? -v : v;
    }
    double ce = 0.0;
    ce = ce + se[0];
    ce = ce + se[1];
    ce = ce + se[2];
    const double bo = b[f];
    const double dt = geo[f].dt;
    const double bn = bo - dt * ce;
    b[f] = bn;
    Rec64 r;
    r.se[0] = se[0]; r.se[1] = se[1]; r.se[2] = se[2];
    r.bz = (bn + bo) * geo[f].inv2A;
    rec[f] = r;
}

void launch_faraday64(cudaStream_t st, int F, const Geo64 *geo, const Topo *topo, const double *e,
                      double *b, Rec64 *rec)
{
    if (F <= 0) return;
    k_faraday64<<<(F + 255) / 256, 256, 0, st>>>(F, geo, topo, e, b, rec);
}

// ------------------------------------------------------------------ push
// 2-D TE specialisation (u_z = 0, E_z = 0, B along z) of the 3-vector
// formulas of Sec. II.C; with u_z = 0 every dropped term is an exact zero,
// so the rounding equals the 3-vector evaluation.

struct Push { double ux, uy, g; };

__device__ __forceinline__ double gam2(double ux, double uy, double ic2)
{
    return sqrt(1.0 + (ux * ux + uy * uy) * ic2);
}

template <int PUSHER>
__device__ __forceinline__ Push push64(double ux, double uy, double Ex, double Ey, double Bz,
                                       double alpha, double c, double ic2)
{
    const double epsx = alpha * Ex, epsy = alpha * Ey;
    const double bz = alpha * Bz;
    const double bb = bz * bz;
    Push out;
    if (PUSHER == FETDPIC_VAY) {
        // Sec. II.C(b): u^n = u^{n-1/2} + eps + v^{n-1/2} x beta; u' = u^n + eps;
        // gamma^{n+1/2} from the quartic; u^{n+1/2} = s (u' + (u'.t) t + u' x t), s = 1/(1+t^2)
        const double g0 = gam2(ux, uy, ic2);
        const double vx = ux / g0, vy = uy / g0;
        const double unx = (ux + epsx) + vy * bz;
        const double uny = (uy + epsy) - vx * bz;
        const double upx = unx + epsx, upy = uny + epsy;
        const double gp = gam2(upx, upy, ic2);
        const double sigma = gp * gp - bb;
        const double gn = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * bb)));
        const double tz = bz / gn;
        const double s = 1.0 / (1.0 + tz * tz);
        out.ux = s * (upx + upy * tz);
        out.uy = s * (upy - upx * tz);
        out.g = gn;
        return out;
    }
    // Boris family, Eqs. (Boris.u1-u4)
    const double umx = ux + epsx, umy = uy + epsy;
    const double gbar = gam2(umx, umy, ic2);                 // Eq. (gamma.middle)
    double tz;
    if (PUSHER == FETDPIC_HC) {
        // Sec. II.C(c): gamma_H from sigma = gamma_B^2 - |beta|^2 (u^- . beta = 0 in 2-D TE)
        const double sigma = gbar * gbar - bb;
        const double gh = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * bb)));
        tz = bz / gh;
    } else if (PUSHER == FETDPIC_BORIS_TAN) {
        const double nb = sqrt(bb);
        tz = (nb == 0.0) ? 0.0 : (bz / nb) * tan(nb / gbar);
    } else {
        tz = bz / gbar;
    }
    const double den = 1.0 + tz * tz;
    const double sz = (2.0 * tz) / den;
    const double uprx = umx + umy * tz, upry = umy - umx * tz;   // u' = u^- + u^- x t
    const double upx = umx + upry * sz, upy = umy - uprx * sz;   // u^+ = u^- + u' x s
    out.ux = upx + epsx;
    out.uy = upy + epsy;
    out.g = gam2(out.ux, out.uy, ic2);
    return out;
}

// --------------------------------------------------------------- deposit

__device__ __forceinline__ void red_add_u64(unsigned long long *p, long long v)
{
    if (v != 0) atomicAdd(p, (unsigned long long)v);
}

// Fixed-point current of one sub-segment, Eq. (I.assign): for local edge m
// with (a, b) = (m+1, m+2), (Q/dt)(l_a^s l_b^f - l_a^f l_b^s), scaled by
// 2^shift/(Q_ref/dt) and rounded to the nearest integer.
__device__ __forceinline__ void seg_current(const double *ls, const double *lf, double w, long long *v)
{
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const int a = (m + 1) % 3, b = (m + 2) % 3;
        const double d = ls[a] * lf[b] - lf[a] * ls[b];
        v[m] = __double2ll_rn(d * w);
    }
}

__device__ __forceinline__ void add_seg(unsigned long long *ifix, const Topo &t, const long long *v)
{
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const long long s = (t.ew[m] & 1) ? -v[m] : v[m];
        red_add_u64(ifix + (t.ew[m] >> 1), s);
    }
}

// --------------------------------------------------------- particle kernel
// One thread per particle.  Blocks never straddle species (species storage
// ranges are padded to 1024).  The first sub-segment of every particle (in
// its starting triangle) is reduced across the warp over runs of equal
// triangle (particles are sorted by triangle), so one lane per run issues the
// three 64-bit integer additions; the rare further sub-segments add directly.
// Integer addition is associative, so the result does not depend on the
// order of particles or atomics: deposits are deterministic.
template <int PUSHER>
__global__ void __launch_bounds__(256) k_particles64(StepArgs64 a)
{
    __shared__ Species S;
    const long long blk = blockIdx.x;
    if (threadIdx.x == 0) S = a.sp[a.blk_sp[blk]];
    __syncthreads();
    const long long p = blk * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int f = a.cell[p];
    const bool live = f >= 0;

    long long v0[3] = {0, 0, 0};
    Topo t0;
    int key = -1;
    bool walking = false;
    // walk state (carried into the divergent continuation)
    double xs = 0, ys = 0, xf = 0, yf = 0, ux = 0, uy = 0, tin = 0.0;
    double lin[3] = {0, 0, 0};
    int min = -1, ncross = 0;
    const double *gxp = nullptr, *gyp = nullptr;
    Topo tc;
    // walk record slot: species storage offset + load index (unmoved by a later sort)
    const long long rp = (a.rec_cap > 0 && live) ? S.off + a.id[p] : 0;

    if (live) {
        const Geo64 &G = a.geo[f];
        tc = a.topo[f];
        const Rec64 R = a.rec[f];
        xs = a.x[p]; ys = a.y[p];
        ux = a.ux[p]; uy = a.uy[p];
        double gx[3], gy[3], X[3], Y[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) { gx[k] = G.gx[k]; gy[k] = G.gy[k]; X[k] = G.X[k]; Y[k] = G.Y[k]; }
        double lam[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int an = (m + 1) % 3;
            lam[m] = gx[m] * (xs - X[an]) + gy[m] * (ys - Y[an]);
        }
        // gather E^n (Sec. II.B): sum_m s_m e_m (l_a grad l_b - l_b grad l_a)
        double Ex = 0.0, Ey = 0.0;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int an = (m + 1) % 3, bn = (m + 2) % 3;
            const double wx = lam[an] * gx[bn] - lam[bn] * gx[an];
            const double wy = lam[an] * gy[bn] - lam[bn] * gy[an];
            Ex = Ex + R.se[m] * wx;
            Ey = Ey + R.se[m] * wy;
        }
        // applied fields: (amplitude x E weight) E_ext, B weight x B_ext in this triangle
        double we = 1.0, wb = 1.0;
        if (a.extw) { const double2 wv = a.extw[f]; we = wv.x; wb = wv.y; }
        const double sa = a.ext_amp[S.inst] * we;
        Ex = Ex + sa * S.ext_ex;
        Ey = Ey + sa * S.ext_ey;
        const double Bz = R.bz + wb * S.ext_bz;
        const Push u = push64<PUSHER>(ux, uy, Ex, Ey, Bz, S.alpha, S.c, S.ic2);
        ux = u.ux; uy = u.uy;
        if (!isfinite(u.g) || !isfinite(ux) || !isfinite(uy)) atomicOr(a.status, (unsigned)ST_NONFINITE);
        const double ig = 1.0 / u.g;
        xf = xs + (ux * ig) * S.dt;                         // Eq. (eq.motion.dis)
        yf = ys + (uy * ig) * S.dt;
        lin[0] = lam[0]; lin[1] = lam[1]; lin[2] = lam[2];

        // first sub-segment, in the starting triangle
        double ls[3], lf[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int an = (m + 1) % 3;
            ls[m] = gx[m] * (xs - X[an]) + gy[m] * (ys - Y[an]);
            lf[m] = gx[m] * (xf - X[an]) + gy[m] * (yf - Y[an]);
        }
        int best = -1;
        double tb = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (lf[k] < 0.0) {
                const double den = ls[k] - lf[k];
                double t = den > 0.0 ? ls[k] / den : tin;
                if (t < tin) t = tin;
                if (best < 0 || t < tb) { best = k; tb = t; }
            }
        }
        t0 = tc;
        key = f;
        if (best < 0) {
            seg_current(lin, lf, S.wfix, v0);
        } else {
            double lout[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) lout[k] = ls[k] + tb * (lf[k] - ls[k]);
            lout[best] = 0.0;
            seg_current(lin, lout, S.wfix, v0);
            walking = true;
            // hand-off (shared with the divergent loop below)
            const int eg = tc.ew[best] >> 1;
            if (ncross >= a.max_cross) {
                xf = xs + tb * (xf - xs); yf = ys + tb * (yf - ys);
                atomicOr(a.status, (unsigned)ST_WALK);
                walking = false;
            } else {
                const int nbw = tc.nb[best];
                if (a.rec_cap > ncross) a.wrec[rp * a.rec_cap + ncross] = nbw < 0 ? -(eg - a.edge_off[S.inst] + 1) : eg - a.edge_off[S.inst];
                ++ncross;
                if (nbw < 0) {
                    const double xw = xs + tb * (xf - xs), yw = ys + tb * (yf - ys);
                    const double gxb = gx[best], gyb = gy[best];
                    const double gg = gxb * gxb + gyb * gyb;
                    const double pr = ((xf - xw) * gxb + (yf - yw) * gyb) / gg;
                    xf = xf - 2.0 * pr * gxb;
                    yf = yf - 2.0 * pr * gyb;
                    const double pu = (ux * gxb + uy * gyb) / gg;
                    ux = ux - 2.0 * pu * gxb;
                    uy = uy - 2.0 * pu * gyb;
                    xs = xw; ys = yw;
                    tin = 0.0;
                    min = best;
                    lin[0] = lout[0]; lin[1] = lout[1]; lin[2] = lout[2];
                } else {
                    const int g2 = nbw >> 2, m2 = nbw & 3;
                    double l2[3];
                    l2[m2] = 0.0;
                    l2[(m2 + 1) % 3] = lout[(best + 2) % 3];
                    l2[(m2 + 2) % 3] = lout[(best + 1) % 3];
                    lin[0] = l2[0]; lin[1] = l2[1]; lin[2] = l2[2];
                    if (a.tshift) {
                        // periodic wall: the rest of the segment continues from the other copy
                        const int sc = a.tshift[3 * f + best];
                        if (sc != 0) {
                            const double2 T = a.period[tc.inst];
                            xs = xs + sc * T.x; ys = ys + sc * T.y;
                            xf = xf + sc * T.x; yf = yf + sc * T.y;
                        }
                    }
                    f = g2;
                    min = m2;
                    tin = tb;
                    tc = a.topo[f];
                }
            }
        }
    }

    // warp segmented reduction of the first sub-segment over runs of equal triangle
    {
        const unsigned full = 0xffffffffu;
        const int kn = __shfl_down_sync(full, key, 1);
        const bool tail = (lane == 31) || (kn != key);
        const unsigned tails = __ballot_sync(full, tail);
        const int seg_end = lane + __ffs(tails >> lane) - 1;
        const int kp = __shfl_up_sync(full, key, 1);
        const bool head = (lane == 0) || (kp != key);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const long long o = __shfl_down_sync(full, v0[m], off);
                if (lane + off <= seg_end) v0[m] += o;
            }
        }
        if (head && key >= 0) add_seg(a.ifix, t0, v0);
    }

    // divergent continuation of the walk (rare: particles that left their triangle)
    while (walking) {
        const Geo64 &G = a.geo[f];
        gxp = G.gx; gyp = G.gy;
        double ls[3], lf[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int an = (m + 1) % 3;
            ls[m] = gxp[m] * (xs - G.X[an]) + gyp[m] * (ys - G.Y[an]);
            lf[m] = gxp[m] * (xf - G.X[an]) + gyp[m] * (yf - G.Y[an]);
        }
        int best = -1;
        double tb = 0.0;
        for (int k = 0; k < 3; ++k) {
            if (k == min) continue;
            if (lf[k] < 0.0) {
                const double den = ls[k] - lf[k];
                double t = den > 0.0 ? ls[k] / den : tin;
                if (t < tin) t = tin;
                if (best < 0 || t < tb) { best = k; tb = t; }
            }
        }
        long long v[3];
        if (best < 0) {
            seg_current(lin, lf, S.wfix, v);
            add_seg(a.ifix, tc, v);
            break;
        }
        double lout[3];
        for (int k = 0; k < 3; ++k) lout[k] = ls[k] + tb * (lf[k] - ls[k]);
        lout[best] = 0.0;
        seg_current(lin, lout, S.wfix, v);
        add_seg(a.ifix, tc, v);
        const int eg = tc.ew[best] >> 1;
        if (ncross >= a.max_cross) {
            xf = xs + tb * (xf - xs); yf = ys + tb * (yf - ys);
            atomicOr(a.status, (unsigned)ST_WALK);
            break;
        }
        const int nbw = tc.nb[best];
        if (a.rec_cap > ncross) a.wrec[rp * a.rec_cap + ncross] = nbw < 0 ? -(eg - a.edge_off[S.inst] + 1) : eg - a.edge_off[S.inst];
        ++ncross;
        if (nbw < 0) {
            const double xw = xs + tb * (xf - xs), yw = ys + tb * (yf - ys);
            const double gxb = gxp[best], gyb = gyp[best];
            const double gg = gxb * gxb + gyb * gyb;
            const double pr = ((xf - xw) * gxb + (yf - yw) * gyb) / gg;
            xf = xf - 2.0 * pr * gxb;
            yf = yf - 2.0 * pr * gyb;
            const double pu = (ux * gxb + uy * gyb) / gg;
            ux = ux - 2.0 * pu * gxb;
            uy = uy - 2.0 * pu * gyb;
            xs = xw; ys = yw;
            tin = 0.0;
            min = best;
            lin[0] = lout[0]; lin[1] = lout[1]; lin[2] = lout[2];
        } else {
            const int g2 = nbw >> 2, m2 = nbw & 3;
            double l2[3];
            l2[m2] = 0.0;
            l2[(m2 + 1) % 3] = lout[(best + 2) % 3];
            l2[(m2 + 2) % 3] = lout[(best + 1) % 3];
            lin[0] = l2[0]; lin[1] = l2[1]; lin[2] = l2[2];
            if (a.tshift) {
                const int sc = a.tshift[3 * f + best];
                if (sc != 0) {
                    const double2 T = a.period[tc.inst];
                    xs = xs + sc * T.x; ys = ys + sc * T.y;
                    xf = xf + sc * T.x; yf = yf + sc * T.y;
                }
            }
            f = g2;
            min = m2;
            tin = tb;
            tc = a.topo[f];
        }
    }

    if (live) {
        a.x[p] = xf; a.y[p] = yf;
        a.ux[p] = ux; a.uy[p] = uy;
        a.cell[p] = f;
        if (a.rec_cap > 0) a.rec_cnt[rp] = ncross;
    }
}

void launch_particles64(cudaStream_t st, int pusher, const StepArgs64 &a)
{
    if (a.nblocks <= 0) return;
    const dim3 grid((unsigned)a.nblocks), block(a.block);
    switch (pusher) {
    case FETDPIC_BORIS: k_particles64<FETDPIC_BORIS><<<grid, block, 0, st>>>(a); break;
    case FETDPIC_BORIS_TAN: k_particles64<FETDPIC_BORIS_TAN><<<grid, block, 0, st>>>(a); break;
    case FETDPIC_VAY: k_particles64<FETDPIC_VAY><<<grid, block, 0, st>>>(a); break;
    default: k_particles64<FETDPIC_HC><<<grid, block, 0, st>>>(a); break;
    }
}

}  // namespace fetdpic

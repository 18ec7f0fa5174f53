// FP32 kernels of the FETD-PIC step: positions are kept cell-local as
// barycentric coordinates (l0, l1; l2 = 1 - l0 - l1), momenta in units of c.
// Gather, push, walk and deposit run in FP32; particles with gamma > 10 take
// the FP64 push (Lorentz factor and momentum update), where FP32 loses the
// 1 - v/c and sigma cancellations.  The field update stays FP64.
#include <cuda_runtime.h>

#include "fetdpic_internal.h"

namespace fetdpic {

// Faraday update in FP64 (in place) and the FP32 field record: in a triangle
// E(lambda) = sum_m s_m e_m (l_a grad l_b - l_b grad l_a) = sum_n l_n V_n with
// V_n = s_{n-1} e_{n-1} grad l_{n+1} - s_{n+1} e_{n+1} grad l_{n-1}; stored
// scaled by dt/(2c) so that q/m times it is alpha E / c.  B_z^n scaled by dt/2.
__global__ void k_faraday32(int F, const Geo64 *__restrict__ geo, const Topo *__restrict__ topo,
                            const double *__restrict__ e, double *__restrict__ b, Rec32 *__restrict__ rec,
                            double c)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const Topo t = topo[f];
    const Geo64 &G = geo[f];
    double se[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const double v = e[t.ew[m] >> 1];
        se[m] = (t.ew[m] & 1) ? -v : v;
    }
    const double bo = b[f];
    const double bn = bo - G.dt * ((se[0] + se[1]) + se[2]);
    b[f] = bn;
    const double s = G.dt / (2.0 * c);
    Rec32 r;
#pragma unroll
    for (int n = 0; n < 3; ++n) {
        const int nm = (n + 2) % 3, np = (n + 1) % 3;
        r.v[2 * n] = (float)(s * (se[nm] * G.gx[np] - se[np] * G.gx[nm]));
        r.v[2 * n + 1] = (float)(s * (se[nm] * G.gy[np] - se[np] * G.gy[nm]));
    }
    r.bz = (float)(0.5 * G.dt * ((bn + bo) * G.inv2A));
    r.pad = 0.f;
    rec[f] = r;
}

void launch_faraday32(cudaStream_t st, int F, const Geo64 *geo, const Topo *topo, const double *e,
                      double *b, Rec32 *rec, double c)
{
    if (F <= 0) return;
    k_faraday32<<<(F + 255) / 256, 256, 0, st>>>(F, geo, topo, e, b, rec, c);
}

// --------------------------------------------------------------- pushers
// Dimensionless (c = 1): eps = alpha E / c, beta = alpha B, u in units of c.

template <int PUSHER, typename T>
__device__ __forceinline__ void push_c1(T &ux, T &uy, T &g, T ex, T ey, T bz)
{
    const T one = T(1), half = T(0.5), two = T(2), four = T(4);
    const T bb = bz * bz;
    if (PUSHER == FETDPIC_VAY) {
        const T g0 = sqrt(one + ux * ux + uy * uy);
        const T vx = ux / g0, vy = uy / g0;
        const T upx = ux + two * ex + vy * bz;
        const T upy = uy + two * ey - vx * bz;
        const T gp2 = one + upx * upx + upy * upy;
        const T sigma = gp2 - bb;
        const T gn = sqrt(half * (sigma + sqrt(sigma * sigma + four * bb)));
        const T tz = bz / gn;
        const T s = one / (one + tz * tz);
        ux = s * (upx + upy * tz);
        uy = s * (upy - upx * tz);
        g = gn;
        return;
    }
    const T umx = ux + ex, umy = uy + ey;
    const T gbar = sqrt(one + umx * umx + umy * umy);
    T tz;
    if (PUSHER == FETDPIC_HC) {
        const T sigma = gbar * gbar - bb;
        const T gh = sqrt(half * (sigma + sqrt(sigma * sigma + four * bb)));
        tz = bz / gh;
    } else if (PUSHER == FETDPIC_BORIS_TAN) {
        const T nb = abs(bz);
        tz = (nb == T(0)) ? T(0) : (bz / nb) * tan(nb / gbar);
    } else {
        tz = bz / gbar;
    }
    const T sz = (two * tz) / (one + tz * tz);
    const T uprx = umx + umy * tz, upry = umy - umx * tz;
    ux = (umx + upry * sz) + ex;
    uy = (umy - uprx * sz) + ey;
    g = sqrt(one + ux * ux + uy * uy);
}

__device__ __forceinline__ void seg_current32(const float *ls, const float *lf, float w, long long *v)
{
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const int a = (m + 1) % 3, b = (m + 2) % 3;
        const float d = ls[a] * lf[b] - lf[a] * ls[b];
        v[m] = __float2ll_rn(d * w);
    }
}

__device__ __forceinline__ void add_seg32(unsigned long long *ifix, const Topo &t, const long long *v)
{
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const long long s = (t.ew[m] & 1) ? -v[m] : v[m];
        if (s != 0) atomicAdd(ifix + (t.ew[m] >> 1), (unsigned long long)s);
    }
}

// Walk step in barycentrics.  The path is r(tau) = r^n + tau * c dt v/c,
// tau in [0, 1]; inside triangle f, l_k(tau) = lin_k + (tau - tin) g_k with
// g_k = G_k . v.  Exit through the edge whose coordinate first reaches 0
// (lowest local index on ties), excluding the entry edge.
__device__ __forceinline__ int exit_edge(const float *lin, const float *g, float tin, int min, float &tb)
{
    int best = -1;
    tb = 2.f;
    const float rem = 1.f - tin;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k == min) continue;
        const float lf = lin[k] + rem * g[k];
        if (lf < 0.f) {
            float t = (g[k] < 0.f) ? tin + lin[k] / (-g[k]) : tin;
            t = fminf(fmaxf(t, tin), 1.f);
            if (best < 0 || t < tb) { best = k; tb = t; }
        }
    }
    return best;
}

template <int PUSHER>
__global__ void __launch_bounds__(256) k_particles32(StepArgs32 a)
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
    float lin[3] = {0.f, 0.f, 0.f}, g[3] = {0.f, 0.f, 0.f};
    float vx = 0.f, vy = 0.f, ux = 0.f, uy = 0.f, gam = 1.f, tin = 0.f;
    float lfin[3] = {0.f, 0.f, 0.f};
    int min = -1, ncross = 0;
    Topo tc;

    if (live) {
        tc = a.topo[f];
        const float4 *rp = reinterpret_cast<const float4 *>(a.rec + f);
        const float4 r0 = rp[0], r1 = rp[1];
        const float4 *gp = reinterpret_cast<const float4 *>(a.geo + f);
        const float4 q0 = gp[0], q1 = gp[1];
        const float G[6] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y};
        const float l0 = a.l0[p], l1 = a.l1[p];
        const float l2 = 1.f - l0 - l1;
        ux = a.ux[p]; uy = a.uy[p];
        // gather (Sec. II.B): alpha E / c = (q/m) sum_n l_n V_n, beta = (q/m) B_z dt/2
        const float ex = S.kappa * (l0 * r0.x + l1 * r0.z + l2 * r1.x) + S.xe_x;
        const float ey = S.kappa * (l0 * r0.y + l1 * r0.w + l2 * r1.y) + S.xe_y;
        const float bz = S.kappa * r1.z + S.xb;
        // push (Sec. II.C); FP64 when gamma > 10
        const float gin2 = 1.f + ux * ux + uy * uy;
        if (gin2 > 100.f) {
            double dux = ux, duy = uy, dg;
            push_c1<PUSHER, double>(dux, duy, dg, (double)ex, (double)ey, (double)bz);
            ux = (float)dux; uy = (float)duy;
            vx = (float)(dux / dg); vy = (float)(duy / dg);
            gam = (float)dg;
        } else {
            push_c1<PUSHER, float>(ux, uy, gam, ex, ey, bz);
            vx = ux / gam; vy = uy / gam;
        }
        if (!isfinite(gam) || !isfinite(ux) || !isfinite(uy)) atomicOr(a.status, (unsigned)ST_NONFINITE);
        // Eq. (eq.motion.dis) in barycentrics: dl_k = c dt grad l_k . v / c
#pragma unroll
        for (int k = 0; k < 3; ++k) g[k] = G[2 * k] * vx + G[2 * k + 1] * vy;
        lin[0] = l0; lin[1] = l1; lin[2] = l2;
        float tb;
        const int best = exit_edge(lin, g, 0.f, -1, tb);
        t0 = tc;
        key = f;
        if (best < 0) {
            lfin[0] = lin[0] + g[0];
            lfin[1] = lin[1] + g[1];
            lfin[2] = 1.f - lfin[0] - lfin[1];
            seg_current32(lin, lfin, S.wfix32, v0);
        } else {
            float lout[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) lout[k] = lin[k] + tb * g[k];
            lout[best] = 0.f;
            seg_current32(lin, lout, S.wfix32, v0);
            walking = true;
            const int eg = tc.ew[best] >> 1;
            if (ncross >= a.max_cross) {
                lfin[0] = lout[0]; lfin[1] = lout[1]; lfin[2] = lout[2];
                atomicOr(a.status, (unsigned)ST_WALK);
                walking = false;
            } else {
                const int nbw = tc.nb[best];
                if (a.rec_cap > ncross) a.wrec[p * a.rec_cap + ncross] = nbw < 0 ? -(eg - a.edge_off[S.inst] + 1) : eg - a.edge_off[S.inst];
                ++ncross;
                if (nbw < 0) {
                    // specular reflection about the wall: normal along G_best
                    const float gxb = G[2 * best], gyb = G[2 * best + 1];
                    const float gg = gxb * gxb + gyb * gyb;
                    const float pu = (ux * gxb + uy * gyb) / gg;
                    ux -= 2.f * pu * gxb; uy -= 2.f * pu * gyb;
                    const float pv = (vx * gxb + vy * gyb) / gg;
                    vx -= 2.f * pv * gxb; vy -= 2.f * pv * gyb;
#pragma unroll
                    for (int k = 0; k < 3; ++k) g[k] = G[2 * k] * vx + G[2 * k + 1] * vy;
                    min = best;
                    lin[0] = lout[0]; lin[1] = lout[1]; lin[2] = lout[2];
                } else {
                    const int m2 = nbw & 3;
                    float l2n[3];
                    l2n[m2] = 0.f;
                    l2n[(m2 + 1) % 3] = lout[(best + 2) % 3];
                    l2n[(m2 + 2) % 3] = lout[(best + 1) % 3];
                    lin[0] = l2n[0]; lin[1] = l2n[1]; lin[2] = l2n[2];
                    f = nbw >> 2;
                    min = m2;
                    tc = a.topo[f];
                    const float4 *gq = reinterpret_cast<const float4 *>(a.geo + f);
                    const float4 w0 = gq[0], w1 = gq[1];
                    g[0] = w0.x * vx + w0.y * vy;
                    g[1] = w0.z * vx + w0.w * vy;
                    g[2] = w1.x * vx + w1.y * vy;
                }
                tin = tb;
            }
        }
    }

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
        if (head && key >= 0) add_seg32(a.ifix, t0, v0);
    }

    while (walking) {
        float tb;
        const int best = exit_edge(lin, g, tin, min, tb);
        long long v[3];
        if (best < 0) {
            const float rem = 1.f - tin;
            lfin[0] = lin[0] + rem * g[0];
            lfin[1] = lin[1] + rem * g[1];
            lfin[2] = 1.f - lfin[0] - lfin[1];
            seg_current32(lin, lfin, S.wfix32, v);
            add_seg32(a.ifix, tc, v);
            break;
        }
        float lout[3];
        const float dtau = tb - tin;
        for (int k = 0; k < 3; ++k) lout[k] = lin[k] + dtau * g[k];
        lout[best] = 0.f;
        seg_current32(lin, lout, S.wfix32, v);
        add_seg32(a.ifix, tc, v);
        const int eg = tc.ew[best] >> 1;
        if (ncross >= a.max_cross) {
            lfin[0] = lout[0]; lfin[1] = lout[1]; lfin[2] = lout[2];
            atomicOr(a.status, (unsigned)ST_WALK);
            break;
        }
        const int nbw = tc.nb[best];
        if (a.rec_cap > ncross) a.wrec[p * a.rec_cap + ncross] = nbw < 0 ? -(eg - a.edge_off[S.inst] + 1) : eg - a.edge_off[S.inst];
        ++ncross;
        const float4 *gq = reinterpret_cast<const float4 *>(a.geo + f);
        if (nbw < 0) {
            const float4 w0 = gq[0], w1 = gq[1];
            const float G[6] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y};
            const float gxb = G[2 * best], gyb = G[2 * best + 1];
            const float gg = gxb * gxb + gyb * gyb;
            const float pu = (ux * gxb + uy * gyb) / gg;
            ux -= 2.f * pu * gxb; uy -= 2.f * pu * gyb;
            const float pv = (vx * gxb + vy * gyb) / gg;
            vx -= 2.f * pv * gxb; vy -= 2.f * pv * gyb;
            for (int k = 0; k < 3; ++k) g[k] = G[2 * k] * vx + G[2 * k + 1] * vy;
            min = best;
            lin[0] = lout[0]; lin[1] = lout[1]; lin[2] = lout[2];
        } else {
            const int m2 = nbw & 3;
            float l2n[3];
            l2n[m2] = 0.f;
            l2n[(m2 + 1) % 3] = lout[(best + 2) % 3];
            l2n[(m2 + 2) % 3] = lout[(best + 1) % 3];
            lin[0] = l2n[0]; lin[1] = l2n[1]; lin[2] = l2n[2];
            f = nbw >> 2;
            min = m2;
            tc = a.topo[f];
            const float4 *gn = reinterpret_cast<const float4 *>(a.geo + f);
            const float4 w0 = gn[0], w1 = gn[1];
            g[0] = w0.x * vx + w0.y * vy;
            g[1] = w0.z * vx + w0.w * vy;
            g[2] = w1.x * vx + w1.y * vy;
        }
        tin = tb;
    }

    if (live) {
        a.l0[p] = lfin[0]; a.l1[p] = lfin[1];
        a.ux[p] = ux; a.uy[p] = uy;
        a.cell[p] = f;
        if (a.rec_cap > 0) a.rec_cnt[p] = ncross;
    }
}

void launch_particles32(cudaStream_t st, int pusher, const StepArgs32 &a)
{
    if (a.nblocks <= 0) return;
    const dim3 grid((unsigned)a.nblocks), block(a.block);
    switch (pusher) {
    case FETDPIC_BORIS: k_particles32<FETDPIC_BORIS><<<grid, block, 0, st>>>(a); break;
    case FETDPIC_BORIS_TAN: k_particles32<FETDPIC_BORIS_TAN><<<grid, block, 0, st>>>(a); break;
    case FETDPIC_VAY: k_particles32<FETDPIC_VAY><<<grid, block, 0, st>>>(a); break;
    default: k_particles32<FETDPIC_HC><<<grid, block, 0, st>>>(a); break;
    }
}

}  // namespace fetdpic

// FP32 kernels of the FETD-PIC step: positions are kept cell-local as
// barycentric coordinates (l0, l1; l2 = 1 - l0 - l1), momenta in units of c.
// Gather, push, walk and deposit run in FP32; particles with gamma > 10 take
// the FP64 push (Lorentz factor and momentum update), where FP32 loses the
// 1 - v/c and sigma cancellations.  The field unknowns and the Faraday update
// stay FP64; the SPAI product of the Ampere update is FP32 (kernels_common.cu).
//
// Built with approximate FP32 division and square root (-prec-div=false
// -prec-sqrt=false, about 2 ulp): the FP32 path is compared with the FP64
// oracle at FP32 round-off tolerances, not bit for bit.
#include <algorithm>

#include <cuda_runtime.h>

#include "fetdpic_internal.h"
#include "field_device.cuh"

namespace fetdpic {

// Faraday update in FP64 (in place) and the FP32 field record: in a triangle
// E(lambda) = sum_m s_m e_m (l_a grad l_b - l_b grad l_a) = sum_n l_n V_n with
// V_n = s_{n-1} e_{n-1} grad l_{n+1} - s_{n+1} e_{n+1} grad l_{n-1}.  Stored
// as dt/(2c) V_n = (s_{n-1} e_{n-1} G_{n+1} - s_{n+1} e_{n+1} G_{n-1}) / (2c^2)
// (G = c dt grad l), so that q/m times it is alpha E / c; B_z^n stored as
// (dt/2) B_z = (dt/2) (b^{n+1/2} + b^{n-1/2}) / (2A).
__device__ __forceinline__ void faraday32_tri(int f, const CstA *__restrict__ csta, const CstB *__restrict__ cstb,
                                              const double2 *__restrict__ dtinv, const double *e, double *b,
                                              Rec32 *rec, float inv2c2, const Ext32 &x, bool ext)
{
    // the triangle's constants are static: loaded before the wait for the kernel that writes e
    const float4 *cp = reinterpret_cast<const float4 *>(csta + f);
    const float4 c0 = __ldg(cp), c1 = __ldg(cp + 1);
    const CstB cb = cstb[f];
    const double2 di = dtinv[f];                    // (dt, 1/(2A))
    pdl_begin();
    // G_2 = -(G_0 + G_1): the barycentric gradients of a triangle sum to zero
    const float G[6] = {c0.x, c0.y, c0.z, c0.w, -(c0.x + c0.z), -(c0.y + c0.w)};
    const int ew[3] = {cb.ew0, __float_as_int(c1.x), __float_as_int(c1.y)};
    double se[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const double v = e[ew[m] >> 1];
        se[m] = (ew[m] & 1) ? -v : v;
    }
    const double bo = b[f];
    const double bn = bo - di.x * ((se[0] + se[1]) + se[2]);
    b[f] = bn;
    float s[3] = {(float)se[0] * inv2c2, (float)se[1] * inv2c2, (float)se[2] * inv2c2};
    Rec32 r;
#pragma unroll
    for (int n = 0; n < 3; ++n) {
        const int nm = (n + 2) % 3, np = (n + 1) % 3;
        r.v[2 * n] = s[nm] * G[2 * np] - s[np] * G[2 * nm];
        r.v[2 * n + 1] = s[nm] * G[2 * np + 1] - s[np] * G[2 * nm + 1];
    }
    double bfield = (bn + bo) * di.y;
    if (ext) {
        // a uniform applied E adds the same value to every node coefficient (sum of lambdas = 1)
        const int k = x.finst[f];
        const ExtField X = x.ext[k];
        double we = 1.0, wb = 1.0;
        if (x.extw) { const double2 wv = x.extw[f]; we = wv.x; wb = wv.y; }
        const double sa = x.amp[k] * we * di.x * x.half_over_c;
        const float ax = (float)(sa * X.ex), ay = (float)(sa * X.ey);
#pragma unroll
        for (int n = 0; n < 3; ++n) { r.v[2 * n] += ax; r.v[2 * n + 1] += ay; }
        bfield += wb * X.bz;                         // B_z = (b^{n+1/2} + b^{n-1/2}) / (2A) + B_ext
    }
    r.bz = (float)(0.5 * di.x * bfield);
    float4 *rp = reinterpret_cast<float4 *>(rec + f);
    rp[0] = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    rp[1] = make_float4(r.v[4], r.v[5], r.bz, __int_as_float(ew[0]));
}

template <bool EXT>
__global__ void __launch_bounds__(256) k_faraday32(int F, const CstA *__restrict__ csta,
                                                   const CstB *__restrict__ cstb,
                                                   const double2 *__restrict__ dtinv,
                                                   const double *__restrict__ e, double *__restrict__ b,
                                                   Rec32 *__restrict__ rec, float inv2c2, Ext32 x)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) { pdl_begin(); return; }
    faraday32_tri(f, csta, cstb, dtinv, e, b, rec, inv2c2, x, EXT);
}

void launch_faraday32(cudaStream_t st, int F, const CstA *csta, const CstB *cstb, const double2 *dtinv,
                      const double *e, double *b, Rec32 *rec, float inv2c2, const Ext32 &x, bool pdl)
{
    if (F <= 0) return;
    const dim3 g((F + 255) / 256);
    if (x.ext) launch_k(pdl, k_faraday32<true>, g, dim3(256), st, F, csta, cstb, dtinv, e, b, rec, inv2c2, x);
    else launch_k(pdl, k_faraday32<false>, g, dim3(256), st, F, csta, cstb, dtinv, e, b, rec, inv2c2, x);
}

// --------------------------------------------------------------- pushers
// Dimensionless (c = 1): eps = alpha E / c, beta = alpha B, u in units of c.
// Returns 1/gamma^{n+1/2} (the position update needs v = u/gamma).

template <typename T> __device__ __forceinline__ T rsqrt_(T x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return 1.0 / sqrt(x); }
template <typename T> __device__ __forceinline__ T rcp_(T x);
template <> __device__ __forceinline__ float rcp_<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double rcp_<double>(double x) { return 1.0 / x; }

// FP64 1/sqrt(x) and 1/x for x in the FP32 normal range: a single-precision
// seed refined by one Newton-Raphson step, y <- y (3 - x y^2) / 2 and
// y <- y (2 - x y).  The relative error squares: at most about 1e-13 for the
// square root (seed within 2.4e-7) and 4e-15 for the reciprocal, against
// IEEE rounding, with a few FP64 operations instead of full-precision
// square-root and division sequences.  Used by the high-gamma push of the FP32
// path, whose results are stored in FP32.
__device__ __forceinline__ double rsqrt_nr(double x)
{
    const double y = (double)rsqrtf((float)x);
    return y * (1.5 - 0.5 * x * (y * y));
}
__device__ __forceinline__ double rcp_nr(double x)
{
    const double y = (double)__frcp_rn((float)x);
    return y * (2.0 - x * y);
}
template <typename T, bool NEWTON> __device__ __forceinline__ T rsq(T x)
{
    if constexpr (NEWTON) return rsqrt_nr(x);
    else return rsqrt_<T>(x);
}
template <typename T, bool NEWTON> __device__ __forceinline__ T rcq(T x)
{
    if constexpr (NEWTON) return rcp_nr(x);
    else return rcp_<T>(x);
}

template <int PUSHER, typename T, bool NEWTON = false>
__device__ __forceinline__ T push_c1(T &ux, T &uy, T ex, T ey, T bz)
{
    const T one = T(1), half = T(0.5), two = T(2), four = T(4);
    const T bb = bz * bz;
    if (PUSHER == FETDPIC_VAY) {
        // Sec. II.C(b): u' = u + 2 eps + v x beta; gamma^{n+1/2} from the quartic root
        // sqrt((sigma + sqrt(sigma^2 + 4|beta|^2))/2); t = beta/gamma; s = 1/(1+t^2)
        const T ig0 = rsq<T, NEWTON>(one + ux * ux + uy * uy);
        const T vx = ux * ig0, vy = uy * ig0;
        const T upx = ux + two * ex + vy * bz;
        const T upy = uy + two * ey - vx * bz;
        const T sigma = one + upx * upx + upy * upy - bb;
        const T r2 = sigma * sigma + four * bb;            // > 0: sigma >= 1 - |beta|^2 + |u'|^2 ...
        const T root = r2 * rsq<T, NEWTON>(r2);
        const T ign = rsq<T, NEWTON>(half * (sigma + root));        // 1/gamma^{n+1/2}
        const T tz = bz * ign;
        const T s = rcq<T, NEWTON>(one + tz * tz);
        ux = s * (upx + upy * tz);
        uy = s * (upy - upx * tz);
        return ign;
    }
    // Boris family, Eqs. (Boris.u1-u4)
    const T umx = ux + ex, umy = uy + ey;
    const T g2 = one + umx * umx + umy * umy;
    T tz;
    if (PUSHER == FETDPIC_HC) {
        // Sec. II.C(c): t = beta / gamma_H, gamma_H^2 = (sigma + sqrt(sigma^2 + 4|beta|^2))/2
        const T sigma = g2 - bb;
        const T r2 = sigma * sigma + four * bb;
        const T root = r2 * rsq<T, NEWTON>(r2);
        tz = bz * rsq<T, NEWTON>(half * (sigma + root));
    } else if (PUSHER == FETDPIC_BORIS_TAN) {
        const T igbar = rsq<T, NEWTON>(g2);
        const T nb = abs(bz);
        tz = (nb == T(0)) ? T(0) : (bz / nb) * tan(nb * igbar);
    } else {
        tz = bz * rsq<T, NEWTON>(g2);
    }
    const T sz = (two * tz) * rcq<T, NEWTON>(one + tz * tz);
    const T uprx = umx + umy * tz, upry = umy - umx * tz;
    ux = (umx + upry * sz) + ex;
    uy = (umy - uprx * sz) + ey;
    return rsq<T, NEWTON>(one + ux * ux + uy * uy);
}

// FP64 push for gamma > 10 (rare; kept out of line so its registers do not
// count against the FP32 main path).  Arguments and result by value, so no
// caller variable needs an address.  Returns (u_x, u_y, v_x, v_y) in units of
// c and 1/gamma.
struct PushOut { float ux, uy, vx, vy, ig; };

template <int PUSHER>
__device__ __noinline__ PushOut push_fp64(float ux, float uy, float ex, float ey, float bz)
{
    double dux = ux, duy = uy;
    const double dig = push_c1<PUSHER, double, true>(dux, duy, (double)ex, (double)ey, (double)bz);
    PushOut o;
    o.ux = (float)dux; o.uy = (float)duy;
    o.vx = (float)(dux * dig); o.vy = (float)(duy * dig);
    o.ig = (float)dig;
    return o;
}

// Fixed-point current of one sub-segment, Eq. (I.assign): round(w (l_a^s l_b^f
// - l_a^f l_b^s)) per local edge m = (a, b) = (m+1, m+2); |w| <= 2^25 - 64 and
// |l_a^s l_b^f - l_a^f l_b^s| <= 1 (to FP32 rounding), so a sum over 64 particles
// fits in 32 bits.
__device__ __forceinline__ void seg_current32(const float *ls, const float *lf, float w, int *v)
{
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const int a = (m + 1) % 3, b = (m + 2) % 3;
        const float d = ls[a] * lf[b] - lf[a] * ls[b];
        v[m] = __float2int_rn(d * w);
    }
}

// Deposit window of a block: fixed-point current of the local edges of the
// triangles [t0, t0 + nt), in global orientation, slot m * WT + (f - t0) for
// local edge m of triangle f.  A value s (|s| < 2^31) goes in as two 32-bit
// shared-memory atomics, its low 16 bits (unsigned) and s >> 16 (signed), so
// s = hi 2^16 + lo exactly; the block adds hi 2^16 + lo of every non-zero slot
// to the global current once, after all its warps are done.  Each addition into
// a slot stands for at least one particle of the block, so with at most 2^16
// particles per block neither sum overflows: sum lo < 2^16 (2^16 - 1) < 2^32,
// |sum hi| <= 2^16 2^15.  Deposits into other triangles, and those of the
// walk, go to the global current directly.  Integer sums: the result is the
// same either way.  nt = 0: no window (every deposit is global).
struct DepWin { unsigned lo, hi; int t0, nt; };        // lo, hi: shared-memory addresses

// Shared-memory reductions, written as such (the window is reached through a
// structure, so a generic atomic would otherwise be possible).
__device__ __forceinline__ void red_shared_u32(unsigned addr, unsigned v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ void red_shared_s32(unsigned addr, int v)
{
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Three integer atomics, issued whatever their value (adding 0 changes nothing,
// and a test would cost a divergent branch per edge).
__device__ __forceinline__ void add_seg32(unsigned long long *ifix, const int *ew, const int *v)
{
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const long long s = (ew[m] & 1) ? -(long long)v[m] : (long long)v[m];
        atomicAdd(ifix + (ew[m] >> 1), (unsigned long long)s);
    }
}

// The deposit of a lane with `dep` set into triangle f, called by the whole
// (converged) warp: into the window when f is in it, else to the global
// current; a warp vote skips a path no lane takes.
template <int WT>
__device__ __forceinline__ void add_seg32w(unsigned long long *ifix, const DepWin &w, bool dep, int f,
                                           const int *ew, const int *v)
{
    if constexpr (WT > 0) {
        const unsigned full = 0xffffffffu;
        const int r = f - w.t0;
        const bool in = dep && (unsigned)r < (unsigned)w.nt;
        if (__any_sync(full, in) && in) {
            const unsigned o = 4u * (unsigned)r;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const int s = (ew[m] & 1) ? -v[m] : v[m];
                red_shared_u32(w.lo + o + 4u * m * WT, (unsigned)s & 0xffffu);
                red_shared_s32(w.hi + o + 4u * m * WT, s >> 16);
            }
        }
        const bool out = dep && !in;
        if (__any_sync(full, out) && out) add_seg32(ifix, ew, v);
    } else {
        if (dep) add_seg32(ifix, ew, v);
    }
}

// Exit edge of the path inside the current triangle: l_k(tau) = lin_k +
// (tau - tin) g_k for tau in [tin, 1].  Candidates are edges k != entry with
// l_k(1) < 0; the exit is the smallest tau_k = tin + lin_k/(-g_k) (lowest k on
// ties), compared by cross-multiplication so only the chosen edge divides.
__device__ __forceinline__ int exit_edge(const float *lin, const float *g, float tin, int min, float &tb)
{
    const float rem = 1.f - tin;
    int best = -1;
    float bn = 0.f, bd = 1.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k == min) continue;
        if (lin[k] + rem * g[k] < 0.f) {
            float num = fmaxf(lin[k], 0.f), den = -g[k];
            if (!(den > 0.f)) { num = 0.f; den = 1.f; }
            if (best < 0 || num * bd < bn * den) { best = k; bn = num; bd = den; }
        }
    }
    tb = best < 0 ? 1.f : fminf(tin + bn / bd, 1.f);
    return best;
}

// Deposit of one sub-segment of a walk: the signed integer current of its entry
// edge `min` gets the carry left by the previous sub-segment on the same edge,
// and the current of its exit edge `best` is carried to the next sub-segment
// instead of being deposited, so a crossed edge takes one atomic, not two.
// Integer sums: the result does not depend on where the additions happen.
__device__ __forceinline__ void add_walk32(unsigned long long *ifix, const int *ew, const int *v, int min,
                                           int best, long long &carry)
{
    const long long cin = carry;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        long long s = (ew[m] & 1) ? -(long long)v[m] : (long long)v[m];
        if (m == min) s += cin;
        if (m == best) carry = s;
        else atomicAdd(ifix + (ew[m] >> 1), (unsigned long long)s);
    }
}

// Register-resident element k (0..2) of a 3-array (no dynamic indexing, so no local memory).
template <typename T>
__device__ __forceinline__ T sel3(const T *a, int k)
{
    return k == 0 ? a[0] : (k == 1 ? a[1] : a[2]);
}

// A particle whose path leaves its starting triangle, queued per warp for the
// walk: its slot, starting triangle and barycentrics, pushed momentum and
// velocity (units of c).
struct __align__(16) WalkItem {
    unsigned p;                  // particle slot (its chunk gives the species)
    int f;                       // starting triangle
    float l0, l1;                // barycentrics at the start of the step (l2 = 1 - l0 - l1)
    float ux, uy, vx, vy;
};
static_assert(sizeof(WalkItem) == 32, "WalkItem layout");

// 32 bytes (32-byte aligned) in one 256-bit load: one L1 wavefront per distinct
// line, where two 128-bit loads of the same bytes take two.
__device__ __forceinline__ void ld_v8(const void *p, float4 &x, float4 &y)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w), "=f"(y.x), "=f"(y.y), "=f"(y.z), "=f"(y.w)
        : "l"(p));
}

// Walk a queued particle along r(tau) = r^n + tau c dt v/c, tau in [0, 1],
// through the triangles it crosses (the current splits the path per triangle,
// Eq. (I.assign)): exit test, deposit of each sub-segment with integer
// atomics, hand-off to the neighbour or specular reflection at a PEC wall, and
// the final particle state.  The particle pass has stored the pushed momentum,
// so it is written again only when a wall reflected it.  Per triangle the walk
// reads 40 bytes in two loads (CstA in one 256-bit load, CstB): a warp of 32
// walkers touches 32 different lines, where one L1 wavefront per line of a
// 256-bit load is half of what two 128-bit loads of the same bytes take.
__device__ __forceinline__ void walk_particle(const StepArgs32 &a, const WalkItem it)
{
    const Sp32 *spp = a.sp + __ldg(a.chunk_sp + (it.p >> 5));
    const float wfix = __ldg(&spp->wfix);
    const int edge_off = __ldg(&spp->edge_off);
    const unsigned p = it.p;
    const long long rp = a.rec_cap > 0 ? (long long)__ldg(&spp->off) + a.id[p] : 0;   // walk record slot
    int f = it.f, ncross = 0, min = -1;
    bool reflected = false;
    float lin[3] = {it.l0, it.l1, 1.f - it.l0 - it.l1};
    float tin = 0.f, ux = it.ux, uy = it.uy, vx = it.vx, vy = it.vy;
    float lfin[3];
    long long carry = 0;                          // current on the entry edge, not yet deposited
    for (;;) {
        float4 c0, c1;
        ld_v8(a.csta + f, c0, c1);
        const int2 cb = __ldg(reinterpret_cast<const int2 *>(a.cstb + f));
        const int ew[3] = {cb.x, __float_as_int(c1.x), __float_as_int(c1.y)};
        float g[3];
        g[0] = c0.x * vx + c0.y * vy;
        g[1] = c0.z * vx + c0.w * vy;
        g[2] = -(g[0] + g[1]);
        float tb;
        const int best = exit_edge(lin, g, tin, min, tb);
        int v[3];
        if (best < 0) {
            const float rem = 1.f - tin;
            lfin[0] = lin[0] + rem * g[0];
            lfin[1] = lin[1] + rem * g[1];
            lfin[2] = 1.f - lfin[0] - lfin[1];
            seg_current32(lin, lfin, wfix, v);
            add_walk32(a.ifix, ew, v, min, -1, carry);
            break;
        }
        float lout[3];
        const float dtau = tb - tin;
#pragma unroll
        for (int k = 0; k < 3; ++k) lout[k] = (k == best) ? 0.f : lin[k] + dtau * g[k];
        seg_current32(lin, lout, wfix, v);
        add_walk32(a.ifix, ew, v, min, best, carry);
        lin[0] = lout[0]; lin[1] = lout[1]; lin[2] = lout[2];
        tin = tb;
        const int eg = sel3(ew, best) >> 1;
        if (ncross >= a.max_cross) {
            atomicAdd(a.ifix + eg, (unsigned long long)carry);
            lfin[0] = lin[0]; lfin[1] = lin[1]; lfin[2] = lin[2];
            atomicOr(a.status, (unsigned)ST_WALK);
            break;
        }
        const int nbw = best == 0 ? __float_as_int(c1.z) : (best == 1 ? __float_as_int(c1.w) : cb.y);
        if (a.rec_cap > ncross) a.wrec[rp * a.rec_cap + ncross] = nbw < 0 ? -(eg - edge_off + 1) : eg - edge_off;
        ++ncross;
        if (nbw < 0) {
            // PEC wall: specular reflection of u and of the rest of the path, normal along G_best
            const float gxb = best == 0 ? c0.x : (best == 1 ? c0.z : -(c0.x + c0.z));
            const float gyb = best == 0 ? c0.y : (best == 1 ? c0.w : -(c0.y + c0.w));
            const float igg = 1.f / (gxb * gxb + gyb * gyb);
            const float pu = (ux * gxb + uy * gyb) * igg;
            ux -= 2.f * pu * gxb; uy -= 2.f * pu * gyb;
            const float pv = (vx * gxb + vy * gyb) * igg;
            vx -= 2.f * pv * gxb; vy -= 2.f * pv * gyb;
            min = best;
            reflected = true;
        } else {
            // hand-off: the neighbour's node m2+1 is our node best+2, its m2+2 our best+1
            const int m2 = nbw & 3;
            const float la = sel3(lin, best == 0 ? 2 : best - 1);
            const float lb = sel3(lin, best == 2 ? 0 : best + 1);
            lin[0] = m2 == 0 ? 0.f : (m2 == 2 ? la : lb);
            lin[1] = m2 == 1 ? 0.f : (m2 == 0 ? la : lb);
            lin[2] = m2 == 2 ? 0.f : (m2 == 1 ? la : lb);
            f = nbw >> 2;
            min = m2;
        }
    }
    a.l0[p] = lfin[0]; a.l1[p] = lfin[1];
    if (reflected) { a.ux[p] = ux; a.uy[p] = uy; }
    a.cell[p] = f;
    if (a.rec_cap > 0) a.rec_cnt[rp] = ncross;
}

constexpr int P32_BLOCK = 256;
constexpr int P32_WARPS = P32_BLOCK / 32;
constexpr int P32_QUEUE = 64;                // walker ring per warp (one particle per lane)

// Particle state of one lane's particle and the records of its triangle:
// r0, r1 = field record (V_0, V_1 | V_2, B_z, edge word 0), c0, c1 = CstA
// (G_0, G_1 | edge words 1, 2, neighbour words 0, 1).
struct PState { int f, sp; float l0, l1, ux, uy; };
struct PRec { float4 r0, r1, c0, c1; };

__device__ __forceinline__ PState load_state(const StepArgs32 &a, unsigned c, int lane)
{
    const unsigned p = c * 32u + (unsigned)lane;
    PState s;
    // streamed once per step: evict-first, so L1 keeps the triangle records
    s.f = __ldcs(a.cell + p); s.l0 = __ldcs(a.l0 + p); s.l1 = __ldcs(a.l1 + p);
    s.ux = __ldcs(a.ux + p); s.uy = __ldcs(a.uy + p);
    s.sp = __ldg(a.chunk_sp + c);
    return s;
}

// The 64 bytes a particle of triangle f needs, in two 256-bit loads.
__device__ __forceinline__ PRec load_rec(const StepArgs32 &a, int f)
{
    // padding slots (f < 0) read triangle 0; their results are discarded
    const int g = f < 0 ? 0 : f;
    PRec r;
    ld_v8(a.rec + g, r.r0, r.r1);
    ld_v8(a.csta + g, r.c0, r.c1);
    return r;
}

// Result of one particle's gather, push and in-triangle test.
struct POne {
    float ux, uy, vx, vy;                    // pushed momentum and velocity (units of c)
    float lf0, lf1;                          // end barycentrics (particles that stay)
    int key;                                 // triangle if it stays, else -1
    bool walking, bad;                       // bad: a live particle's velocity is not finite
    int v[3];                                // fixed-point current if it stays, else 0
};

// Gather (Sec. II.B), push (Sec. II.C; FP64 when gamma > 10), move in
// barycentrics (Eq. (eq.motion.dis): dl_k = c dt grad l_k . v/c, with
// dl_2 = -(dl_0 + dl_1) so the barycentrics keep summing to 1), and the
// current of a particle that stays in its triangle (Eq. (I.assign), written
// i_ab += (Q/dt)(l_a dl_b - dl_a l_b)).
template <int PUSHER>
__device__ __forceinline__ POne one_particle(float kappa, float wfix, int f, float l0, float l1, float ux,
                                             float uy, const PRec &r)
{
    POne o;
    const bool live = f >= 0;
    const float l2 = 1.f - l0 - l1;
    // alpha E / c = (q/m) sum_n l_n V_n, beta = (q/m) B_z dt/2
    const float ex = kappa * (l0 * r.r0.x + l1 * r.r0.z + l2 * r.r1.x);
    const float ey = kappa * (l0 * r.r0.y + l1 * r.r0.w + l2 * r.r1.y);
    const float bz = kappa * r.r1.z;
    float ig, vx, vy;
    if (1.f + ux * ux + uy * uy > 100.f) {
        const PushOut q = push_fp64<PUSHER>(ux, uy, ex, ey, bz);
        ux = q.ux; uy = q.uy; vx = q.vx; vy = q.vy; ig = q.ig;
    } else {
        ig = push_c1<PUSHER, float>(ux, uy, ex, ey, bz);
        vx = ux * ig; vy = uy * ig;
    }
    o.bad = live && !isfinite(vx + vy);
    const float g0 = r.c0.x * vx + r.c0.y * vy;
    const float g1 = r.c0.z * vx + r.c0.w * vy;
    const float g2 = -(g0 + g1);
    const float lf0 = l0 + g0, lf1 = l1 + g1;
    const bool stays = lf0 >= 0.f && lf1 >= 0.f && l2 + g2 >= 0.f;
    const float wk = (live && stays) ? wfix : 0.f;
    o.v[0] = __float2int_rn((l1 * g2 - g1 * l2) * wk);
    o.v[1] = __float2int_rn((l2 * g0 - g2 * l0) * wk);
    o.v[2] = __float2int_rn((l0 * g1 - g0 * l1) * wk);
    o.ux = ux; o.uy = uy; o.vx = vx; o.vy = vy; o.lf0 = lf0; o.lf1 = lf1;
    o.key = (live && stays) ? f : -1;
    o.walking = live && !stays;
    return o;
}

__device__ __forceinline__ WalkItem walk_item(unsigned p, int f, int sp, float l0, float l1, const POne &o)
{
    WalkItem it;
    (void)sp;
    it.p = p; it.f = f;
    it.l0 = l0; it.l1 = l1;
    it.ux = o.ux; it.uy = o.uy; it.vx = o.vx; it.vy = o.vy;
    return it;
}

// Ring slot of this lane's walker (ring positions are warp-uniform); advances qtail.
__device__ __forceinline__ unsigned ring_slot(unsigned &qtail, bool walking, int lane)
{
    const unsigned wm = __ballot_sync(0xffffffffu, walking);
    const unsigned slot = qtail + __popc(wm & ((1u << lane) - 1u));
    qtail += __popc(wm);
    return slot;
}

// Segmented sum of v over runs of equal key across the warp (keys of a run are
// adjacent: the particles are sorted by triangle); the run heads deposit the
// sums with three integer atomics.  (tests/test_run_reduction_model.py replays
// this reduction, with the two-particle kernel's hand-off of first particles,
// lane by lane on random warps.)
template <int WT = 0>
__device__ __forceinline__ void run_deposit(unsigned long long *ifix, int key, int *v, int lane, const int *ew,
                                            const DepWin &w = DepWin{})
{
    const unsigned full = 0xffffffffu;
    const int kn = __shfl_down_sync(full, key, 1);
    const unsigned tails = __ballot_sync(full, (lane == 31) || (kn != key));
    const int seg_end = lane + __ffs(tails >> lane) - 1;
    const int kp = __shfl_up_sync(full, key, 1);
    const bool head = (lane == 0) || (kp != key);
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
        const int o0 = __shfl_down_sync(full, v[0], off);
        const int o1 = __shfl_down_sync(full, v[1], off);
        const int o2 = __shfl_down_sync(full, v[2], off);
        if (lane + off <= seg_end) { v[0] += o0; v[1] += o1; v[2] += o2; }
    }
    // the levels 4, 8, 16 only when some run spans more lanes than that (a warp vote):
    // sorted runs are about 10 lanes long, and drifted particles make them shorter
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
        if (!__any_sync(full, seg_end - lane >= off)) break;
        const int o0 = __shfl_down_sync(full, v[0], off);
        const int o1 = __shfl_down_sync(full, v[1], off);
        const int o2 = __shfl_down_sync(full, v[2], off);
        if (lane + off <= seg_end) { v[0] += o0; v[1] += o1; v[2] += o2; }
    }
    add_seg32w<WT>(ifix, w, head && key >= 0, key, ew, v);
}

// One 32-particle chunk, one particle per lane: gather, push, in-triangle
// test, current of the particles that stay (run deposit), state stores;
// walkers go to the warp's ring, which is walked 32 at a time.
template <int PUSHER>
__device__ __forceinline__ void process_chunk(const StepArgs32 &a, unsigned c, int lane, const PState &s,
                                              const PRec &r, WalkItem *q, unsigned &qhead, unsigned &qtail)
{
    const unsigned p = c * 32u + (unsigned)lane;
    const Sp32 *spp = a.sp + s.sp;
    const float2 kw = __ldg(reinterpret_cast<const float2 *>(spp));      // q/m, fixed-point weight
    POne o = one_particle<PUSHER>(kw.x, kw.y, s.f, s.l0, s.l1, s.ux, s.uy, r);
    if (o.bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
    {
        const unsigned slot = ring_slot(qtail, o.walking, lane);
        if (o.walking) q[slot & (P32_QUEUE - 1)] = walk_item(p, s.f, s.sp, s.l0, s.l1, o);
    }
    {
        const int ew[3] = {__float_as_int(r.r1.w), __float_as_int(r.c1.x), __float_as_int(r.c1.y)};
        run_deposit(a.ifix, o.key, o.v, lane, ew);
    }
    if (o.key >= 0) {
        __stcs(a.l0 + p, o.lf0); __stcs(a.l1 + p, o.lf1);
        if (a.rec_cap > 0) a.rec_cnt[__ldg(&spp->off) + a.id[p]] = 0;
    }
    if (s.f >= 0) { __stcs(a.ux + p, o.ux); __stcs(a.uy + p, o.uy); }
    if (qtail - qhead >= 32) {
        __syncwarp();
        const WalkItem w = q[(qhead + lane) & (P32_QUEUE - 1)];
        walk_particle(a, w);
        qhead += 32;
        __syncwarp();
    }
}

template <int QN>
__device__ __forceinline__ void drain(const StepArgs32 &a, WalkItem *q, unsigned qhead, unsigned qtail, int lane)
{
    const unsigned left = qtail - qhead;
    if (left > 0) {
        __syncwarp();
        if ((unsigned)lane < left) walk_particle(a, q[(qhead + lane) & (QN - 1)]);
    }
}

// Persistent kernel: each warp takes a contiguous range of 32-particle chunks
// (consecutive chunks of sorted particles share triangles, so their records
// come from L1); the next chunk's particle state is loaded into registers
// while the current one is processed.  MINB only sets the register budget.
// Species ranges are padded to 1024, so a chunk never straddles species.
// Integer sums are exact and every variant runs the same per-particle code,
// so the result depends on neither MINB nor particle, queue or atomic order.
template <int PUSHER, int MINB, int NW>
__global__ void __launch_bounds__(NW * 32, MINB) k_particles32(StepArgs32 a)
{
    pdl_begin();
    __shared__ WalkItem qbuf[NW][P32_QUEUE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WalkItem *q = qbuf[warp];
    unsigned qhead = 0, qtail = 0;                    // warp-uniform ring positions
    const unsigned nwarps = gridDim.x * NW;
    const unsigned wid = blockIdx.x * NW + warp;
    const unsigned K = (unsigned)((a.nchunks + nwarps - 1) / nwarps);
    unsigned c = wid * K;
    const unsigned cend = (unsigned)min((long long)c + K, a.nchunks);
    if (c >= cend) return;
    PState sn = load_state(a, c, lane);
    for (; c < cend; ++c) {
        const PState s = sn;
        if (c + 1 < cend) sn = load_state(a, c + 1, lane);
        const PRec r = load_rec(a, s.f);
        process_chunk<PUSHER>(a, c, lane, s, r, q, qhead, qtail);
    }
    drain<P32_QUEUE>(a, q, qhead, qtail, lane);
}

// ------------------------------------------------- two particles per lane
// Each lane takes two adjacent particles, so a warp chunk is 64 particles and
// the state moves in 8-byte vector loads and stores.  When both particles of
// a lane are in the same triangle their currents are summed in the lane, so
// the warp-segmented reduction runs once per 64 particles; a lane whose pair
// straddles a change of triangle hands its first particle to the previous
// lane's run (or deposits it with its own integer atomics when that run is
// another triangle's).  The per-particle arithmetic is one_particle's, as in
// the one-particle-per-lane kernel.
constexpr int P32_QUEUE2 = 128;              // walker ring per warp: 31 pending + 64 new fit

struct PState2 { int fa, fb, sp; float2 l0, l1, ux, uy; };

__device__ __forceinline__ PState2 load_state2(const StepArgs32 &a, unsigned c, int lane)
{
    const unsigned p = c * 64u + 2u * (unsigned)lane;
    PState2 s;
    const int2 f = __ldcs(reinterpret_cast<const int2 *>(a.cell + p));
    s.fa = f.x; s.fb = f.y;
    s.l0 = __ldcs(reinterpret_cast<const float2 *>(a.l0 + p));
    s.l1 = __ldcs(reinterpret_cast<const float2 *>(a.l1 + p));
    s.ux = __ldcs(reinterpret_cast<const float2 *>(a.ux + p));
    s.uy = __ldcs(reinterpret_cast<const float2 *>(a.uy + p));
    s.sp = __ldg(a.chunk_sp + 2 * c);
    return s;
}

// SEQ: the second particle's records are loaded after the first particle's
// arithmetic (a compiler barrier keeps them there), so the two record sets are
// never live together; when both particles share a triangle the second load
// hits L1.
template <int PUSHER, bool SEQ, int WT>
__device__ __forceinline__ void process_chunk2(const StepArgs32 &a, unsigned c, int lane, const PState2 &s,
                                               const PRec &ra, const PRec &rb_in, WalkItem *q, unsigned &qhead,
                                               unsigned &qtail, bool &bad, const DepWin &dw)
{
    const unsigned full = 0xffffffffu;
    const unsigned pa = c * 64u + 2u * (unsigned)lane;
    const Sp32 *spp = a.sp + s.sp;
    const float2 kw = __ldg(reinterpret_cast<const float2 *>(spp));      // q/m, fixed-point weight
    const POne A = one_particle<PUSHER>(kw.x, kw.y, s.fa, s.l0.x, s.l1.x, s.ux.x, s.uy.x, ra);
    {
        const unsigned slot = ring_slot(qtail, A.walking, lane);
        if (A.walking) q[slot & (P32_QUEUE2 - 1)] = walk_item(pa, s.fa, s.sp, s.l0.x, s.l1.x, A);
    }
    const int ewa[3] = {__float_as_int(ra.r1.w), __float_as_int(ra.c1.x), __float_as_int(ra.c1.y)};
    PRec rb;
    if (SEQ) {
        asm volatile("" ::: "memory");
        rb = load_rec(a, s.fb);
    } else {
        rb = rb_in;
    }
    const POne B = one_particle<PUSHER>(kw.x, kw.y, s.fb, s.l0.y, s.l1.y, s.ux.y, s.uy.y, rb);
    {
        const unsigned slot = ring_slot(qtail, B.walking, lane);
        if (B.walking) q[slot & (P32_QUEUE2 - 1)] = walk_item(pa + 1, s.fb, s.sp, s.l0.y, s.l1.y, B);
    }
    bad |= A.bad | B.bad;
    // current of the particles that stay, Eq. (I.assign).  The run of a
    // thread's second particle is reduced across the warp; a first particle that ends a
    // different run (an "orphan") is handed to the previous thread when that thread's second
    // particle lies in the same triangle, and deposits with its own atomics otherwise.
    const bool same = A.key == B.key;
    const int key = B.key;
    const int okey = same ? -1 : A.key;                  // orphan's triangle, -1: none
    const int kp = __shfl_up_sync(full, key, 1);
    const bool given = lane > 0 && okey >= 0 && okey == kp;
    add_seg32w<WT>(a.ifix, dw, okey >= 0 && !given, okey, ewa, A.v);
    int v0[3];
    {
        const bool taken = __shfl_down_sync(full, given, 1) && lane < 31;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int on = __shfl_down_sync(full, A.v[m], 1);        // next thread's orphan
            v0[m] = B.v[m] + (same ? A.v[m] : 0) + (taken ? on : 0);
        }
    }
    {
        const int ewb[3] = {__float_as_int(rb.r1.w), __float_as_int(rb.c1.x), __float_as_int(rb.c1.y)};
        run_deposit<WT>(a.ifix, key, v0, lane, ewb, dw);
    }
    // state: both slots of every lane are written.  A walker's position is rewritten by its
    // walk after the warp barrier below, and its momentum (stored here as pushed) only if a
    // wall reflects it; a padding slot (triangle -1) is never read, so it takes whatever
    // was computed for it.
    const bool sa = A.key >= 0, sb = B.key >= 0;
    __stcs(reinterpret_cast<float2 *>(a.l0 + pa), make_float2(A.lf0, B.lf0));
    __stcs(reinterpret_cast<float2 *>(a.l1 + pa), make_float2(A.lf1, B.lf1));
    __stcs(reinterpret_cast<float2 *>(a.ux + pa), make_float2(A.ux, B.ux));
    __stcs(reinterpret_cast<float2 *>(a.uy + pa), make_float2(A.uy, B.uy));
    if (a.rec_cap > 0) {
        const int off = __ldg(&spp->off);
        if (sa) a.rec_cnt[off + a.id[pa]] = 0;
        if (sb) a.rec_cnt[off + a.id[pa + 1]] = 0;
    }
    while (qtail - qhead >= 32) {
        __syncwarp();
        const WalkItem w = q[(qhead + lane) & (P32_QUEUE2 - 1)];
        walk_particle(a, w);
        qhead += 32;
        __syncwarp();
    }
}

// WT > 0: the block's deposit window holds WT triangles centred on the
// triangle of the particle in the middle of the block's chunk range (the warps
// of a block take adjacent ranges of sorted particles, so their triangles, in
// Hilbert order, are a compact patch of the mesh; the window also catches most
// particles that have moved to a neighbour since the sort).
template <int PUSHER, int MINB, int NW, bool SEQ, int WT = 0>
__global__ void __launch_bounds__(NW * 32, MINB) k_particles32x2(StepArgs32 a)
{
    __shared__ WalkItem qbuf[NW][P32_QUEUE2];
    __shared__ unsigned wlo[WT > 0 ? 3 * WT : 1];
    __shared__ int whi[WT > 0 ? 3 * WT : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WalkItem *q = qbuf[warp];
    unsigned qhead = 0, qtail = 0;
    const unsigned nwarps = gridDim.x * NW;
    const unsigned wid = blockIdx.x * NW + warp;
    const long long n64 = a.nchunks / 2;         // species ranges are padded to 1024, so nchunks is even
    const unsigned K = (unsigned)((n64 + nwarps - 1) / nwarps);
    unsigned c = wid * K;
    const unsigned cend = (unsigned)min((long long)c + K, n64);
    PState2 sn;
    if (c < cend) sn = load_state2(a, c, lane);            // in flight while the window is set up
    DepWin dw{(unsigned)__cvta_generic_to_shared(wlo), (unsigned)__cvta_generic_to_shared(whi), 0, 0};
    if (WT > 0) {
        for (int i = threadIdx.x; i < 3 * WT; i += NW * 32) { wlo[i] = 0u; whi[i] = 0; }
        const long long b0 = (long long)blockIdx.x * NW * K, b1 = min(b0 + (long long)NW * K, n64);
        int tc = -1;
        if (b0 < b1 && (long long)NW * K * 64 <= 65536) {       // the window's sums cannot overflow
            tc = a.cell[((b0 + b1) / 2) * 64];
            if (tc < 0) tc = a.cell[b0 * 64];            // middle chunk in a species' padding
        }
        dw.t0 = tc - WT / 2;
        dw.nt = tc >= 0 ? WT : 0;
        __syncthreads();
    }
    // Only the field records come from the kernel this one may overlap (Faraday); the
    // particle state and the cleared current were written before Faraday started, so the
    // first state load and the window set-up go ahead of the wait.
    pdl_begin();
    if (c < cend) {
        bool bad = false;
        for (; c < cend; ++c) {
            const PState2 s = sn;
            if (c + 1 < cend) sn = load_state2(a, c + 1, lane);
            const PRec ra = load_rec(a, s.fa);
            PRec rb;
            if (!SEQ) rb = load_rec(a, s.fb);
            process_chunk2<PUSHER, SEQ, WT>(a, c, lane, s, ra, rb, q, qhead, qtail, bad, dw);
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ST_NONFINITE);
        drain<P32_QUEUE2>(a, q, qhead, qtail, lane);
    }
    if constexpr (WT > 0) {
        // a non-zero slot belongs to a triangle some particle was deposited in, so t is valid;
        // all edge words are loaded before the first atomic, so the flush waits for one load
        constexpr int NIT = 3 * WT / (NW * 32);
        static_assert(NIT * NW * 32 == 3 * WT, "window slots per thread");
        __syncthreads();
        long long v[NIT];
        int ew[NIT];
#pragma unroll
        for (int k = 0; k < NIT; ++k) {
            const int i = threadIdx.x + k * NW * 32;
            v[k] = (long long)whi[i] * 65536 + (long long)wlo[i];
            const int m = i / WT, t = dw.t0 + (i - m * WT);
            ew[k] = 0;
            if (v[k] != 0)
                ew[k] = m == 0 ? __ldg(&a.cstb[t].ew0) : (m == 1 ? __ldg(&a.csta[t].ew1) : __ldg(&a.csta[t].ew2));
        }
#pragma unroll
        for (int k = 0; k < NIT; ++k)
            if (v[k] != 0) atomicAdd(a.ifix + (ew[k] >> 1), (unsigned long long)v[k]);
    }
}

// ------------------------------------------------------- staged variant
// Particle state streamed into shared memory by bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier), ST_DEPTH chunks ahead of the
// chunk being processed: one lane per warp issues five 128-byte copies per
// chunk (cell, l0, l1, ux, uy), so the bytes in flight no longer depend on the
// registers a thread can spare.  Every wait on an mbarrier is bounded; a wait
// that gives up (after StepArgs32::spin polls) sets ST_TIMEOUT and the warp
// stops after waiting, with the fixed bound ST_SPIN, for the copies it still
// has in flight, so no copy lands in shared memory the block no longer owns.
constexpr int ST_DEPTH = 4;
constexpr unsigned ST_SPIN = 1u << 22;

struct __align__(16) StageBuf {
    int cell[32];
    float l0[32], l1[32], ux[32], uy[32];
};

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_to_smem(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Non-blocking test of phase `parity` (test_wait returns at once; try_wait may
// suspend the thread for a hardware-chosen time, which would make the poll
// count of a bounded wait meaningless).
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned limit)
{
    for (unsigned k = 0; k < limit; ++k)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// Lane 0 of the warp: start the copies of chunk c into stage buffer `b`.
__device__ __forceinline__ void stage_issue(const StepArgs32 &a, unsigned c, StageBuf *b, unsigned long long *bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // earlier reads of this buffer first
    mbar_expect_tx(bar, 5 * 128);
    const size_t o = (size_t)c * 32;
    bulk_to_smem(b->cell, a.cell + o, 128, bar);
    bulk_to_smem(b->l0, a.l0 + o, 128, bar);
    bulk_to_smem(b->l1, a.l1 + o, 128, bar);
    bulk_to_smem(b->ux, a.ux + o, 128, bar);
    bulk_to_smem(b->uy, a.uy + o, 128, bar);
}

template <int PUSHER>
__global__ void __launch_bounds__(P32_BLOCK, 3) k_particles32_staged(StepArgs32 a)
{
    pdl_begin();
    __shared__ WalkItem qbuf[P32_WARPS][P32_QUEUE];
    __shared__ StageBuf sbuf[P32_WARPS][ST_DEPTH];
    __shared__ unsigned long long sbar[P32_WARPS][ST_DEPTH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WalkItem *q = qbuf[warp];
    StageBuf *buf = sbuf[warp];
    unsigned long long *bar = sbar[warp];
    unsigned qhead = 0, qtail = 0;
    const unsigned nwarps = gridDim.x * P32_WARPS;
    const unsigned wid = blockIdx.x * P32_WARPS + warp;
    const unsigned K = (unsigned)((a.nchunks + nwarps - 1) / nwarps);
    const unsigned c0 = wid * K;
    const unsigned cend = (unsigned)min((long long)c0 + K, a.nchunks);
    if (c0 >= cend) return;
    if (lane == 0) {
        for (int s = 0; s < ST_DEPTH; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (lane == 0)
        for (int s = 0; s < ST_DEPTH; ++s)
            if (c0 + s < cend) stage_issue(a, c0 + s, &buf[s], &bar[s]);
    __syncwarp();
    unsigned phase = 0;                               // bit s = parity to wait for on stage s
    unsigned inflight = 0;                            // bit s = stage s has copies in flight
    for (int s = 0; s < ST_DEPTH; ++s)
        if (c0 + s < cend) inflight |= 1u << s;
    int spn = a.chunk_sp[c0];
    bool ok = true;
    for (unsigned c = c0; c < cend; ++c) {
        const int s = (int)((c - c0) % ST_DEPTH);
        const int sp = spn;
        if (c + 1 < cend) spn = a.chunk_sp[c + 1];
        // all lanes poll; the warp gives up together so no lane is left in a full-mask shuffle
        if (!__all_sync(0xffffffffu, mbar_wait(&bar[s], (phase >> s) & 1u, a.spin))) { ok = false; break; }
        phase ^= 1u << s;
        inflight &= ~(1u << s);
        PState st;
        st.f = buf[s].cell[lane]; st.l0 = buf[s].l0[lane]; st.l1 = buf[s].l1[lane];
        st.ux = buf[s].ux[lane]; st.uy = buf[s].uy[lane]; st.sp = sp;
        __syncwarp();
        if (c + ST_DEPTH < cend) {
            if (lane == 0) stage_issue(a, c + ST_DEPTH, &buf[s], &bar[s]);
            inflight |= 1u << s;
        }
        const PRec r = load_rec(a, st.f);
        process_chunk<PUSHER>(a, c, lane, st, r, q, qhead, qtail);
    }
    if (!ok) {
        if (lane == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
        // let the copies still in flight land before the block's shared memory goes away
        for (int s = 0; s < ST_DEPTH; ++s)
            if (inflight & (1u << s)) mbar_wait(&bar[s], (phase >> s) & 1u, ST_SPIN);
        return;
    }
    drain<P32_QUEUE>(a, q, qhead, qtail, lane);
}

// Persistent grid: resident blocks per SM (from the occupancy calculator) times
// the SM count, capped by the work.  MINB = minimum resident blocks per SM the
// register allocation targets (2, 3 or 4 x 256 threads); chosen by `variant`.
template <int PUSHER, int MINB, int NW = P32_WARPS>
static void launch_p32(cudaStream_t st, const StepArgs32 &a)
{
    static int per_sm = 0, sms = 0, dev = -1;
    int d = 0;
    cudaGetDevice(&d);
    if (d != dev || per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_particles32<PUSHER, MINB, NW>, NW * 32, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        dev = d;
        if (per_sm < 1) per_sm = 1;
    }
    const long long need = (a.nchunks + NW - 1) / NW;
    const long long grid = std::min<long long>(need, (long long)per_sm * sms);
    if (grid <= 0) return;
    launch_k(a.pdl, k_particles32<PUSHER, MINB, NW>, dim3((unsigned)grid), dim3(NW * 32), st, a);
}

template <int PUSHER, int MINB, int NW, bool SEQ = false, int WT = 0>
static void launch_p32x2(cudaStream_t st, const StepArgs32 &a)
{
    static int per_sm = 0, sms = 0, dev = -1;
    int d = 0;
    cudaGetDevice(&d);
    if (d != dev || per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_particles32x2<PUSHER, MINB, NW, SEQ, WT>, NW * 32, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        dev = d;
        if (per_sm < 1) per_sm = 1;
    }
    const long long need = (a.nchunks / 2 + NW - 1) / NW;
    const long long grid = std::min<long long>(need, (long long)per_sm * sms);
    if (grid <= 0) return;
    launch_k(a.pdl, k_particles32x2<PUSHER, MINB, NW, SEQ, WT>, dim3((unsigned)grid), dim3(NW * 32), st, a);
}

template <int PUSHER>
static void launch_p32s(cudaStream_t st, const StepArgs32 &a)
{
    static int per_sm = 0, sms = 0, dev = -1;
    int d = 0;
    cudaGetDevice(&d);
    if (d != dev || per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_particles32_staged<PUSHER>, P32_BLOCK, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        dev = d;
        if (per_sm < 1) per_sm = 1;
    }
    const long long need = (a.nchunks + P32_WARPS - 1) / P32_WARPS;
    const long long grid = std::min<long long>(need, (long long)per_sm * sms);
    if (grid <= 0) return;
    launch_k(a.pdl, k_particles32_staged<PUSHER>, dim3((unsigned)grid), dim3(P32_BLOCK), st, a);
}

template <int PUSHER>
static void launch_p32v(cudaStream_t st, const StepArgs32 &a)
{
    switch (a.variant) {
    case 5: launch_p32s<PUSHER>(st, a); break;
    case 6: launch_p32<PUSHER, 7, 4>(st, a); break;
    case 7: launch_p32<PUSHER, 14, 2>(st, a); break;
    case 8: launch_p32x2<PUSHER, 2, 8>(st, a); break;
    case 9: launch_p32x2<PUSHER, 5, 4>(st, a); break;
    case 10: launch_p32x2<PUSHER, 10, 2>(st, a); break;
    case 11: launch_p32x2<PUSHER, 6, 4, true>(st, a); break;
    case 12: launch_p32x2<PUSHER, 12, 2, true>(st, a); break;
    case 19: launch_p32x2<PUSHER, 14, 2, true>(st, a); break;
    case 20: launch_p32x2<PUSHER, 12, 2, true, 256>(st, a); break;
    case 13: launch_p32x2<PUSHER, 10, 2, false, 320>(st, a); break;
    case 14: launch_p32x2<PUSHER, 10, 2, false, 256>(st, a); break;
    case 15: launch_p32x2<PUSHER, 12, 2, true, 192>(st, a); break;
    case 16: launch_p32x2<PUSHER, 5, 4, false, 640>(st, a); break;
    case 2: launch_p32<PUSHER, 2>(st, a); break;
    case 4: launch_p32<PUSHER, 4>(st, a); break;
    default: launch_p32<PUSHER, 3>(st, a); break;     // measured best on GB300 (no spills, 24 warps/SM)
    }
}

void launch_particles32(cudaStream_t st, int pusher, const StepArgs32 &a)
{
    if (a.nchunks <= 0) return;
    switch (pusher) {
    case FETDPIC_BORIS: launch_p32v<FETDPIC_BORIS>(st, a); break;
    case FETDPIC_BORIS_TAN: launch_p32v<FETDPIC_BORIS_TAN>(st, a); break;
    case FETDPIC_VAY: launch_p32v<FETDPIC_VAY>(st, a); break;
    default: launch_p32v<FETDPIC_HC>(st, a); break;
    }
}

}  // namespace fetdpic

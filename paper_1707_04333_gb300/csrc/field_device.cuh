// Device code shared by the field-update kernels and the fused FP32 step:
// cache-policy loads of static operands, the per-edge curl of Ampere's law,
// and a bounded grid-wide barrier for cooperative launches.
#pragma once

#include <cuda_runtime.h>

#include "fetdpic_internal.h"

namespace fetdpic {

// Static field-update operands (the SPAI in sliced ELL, per-edge face pairs and
// coefficients) are read once per step while hundreds of MB of particle state
// stream through L2 between two reads: they are loaded with an L2 evict-last
// policy so the streaming state, not they, is what L2 drops.
__device__ __forceinline__ unsigned long long l2_keep()
{
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
template <typename T> __device__ __forceinline__ T ld_keep(const T *p, unsigned long long pol);
template <> __device__ __forceinline__ int ld_keep<int>(const int *p, unsigned long long pol)
{
    int v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ float ld_keep<float>(const float *p, unsigned long long pol)
{
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ double ld_keep<double>(const double *p, unsigned long long pol)
{
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ int2 ld_keep<int2>(const int2 *p, unsigned long long pol)
{
    int2 v;
    asm("ld.global.nc.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ double2 ld_keep<double2>(const double2 *p, unsigned long long pol)
{
    double2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
    return v;
}

// r = C^T [*mu^-1] b^{n+1/2} - i^{n+1/2} on edge e (Eq. (semi.dis.curl.2)),
// with [*mu^-1] = 1/(mu0 A_f) folded into ecoef = s_f/(mu0 A_f).  The
// fixed-point current is converted (unit = (q_ref/dt) 2^-shift per
// instance), kept in j for reading, and cleared for the next step.  The dual
// flux d += dt r accumulates for the Gauss-law check (d == NULL: checks off);
// r (FP64) is stored for the FP64 SpMV, r32 for the FP32 one (either NULL).
__device__ __forceinline__ void curl_h_edge(const AmpereArgs &a, int e, unsigned long long keep)
{
    const int2 fa = ld_keep(a.efac + e, keep);
    const double2 cf = ld_keep(a.ecoef + e, keep);
    double h = a.b[fa.x] * cf.x;
    if (fa.y >= 0) h += a.b[fa.y] * cf.y;
    const int in = ld_keep(a.einst + e, keep);
    const long long iv = (long long)a.ifix[e];
    a.ifix[e] = 0ull;
    const double cur = (double)iv * a.inst_unit[in];
    const double rv = h - cur;
    if (a.r) a.r[e] = rv;
    if (a.r32) a.r32[e] = (float)rv;
    a.j[e] = cur;
    if (a.d) a.d[e] += a.inst_dt[in] * rv;
}

// Grid-wide barrier of a cooperative launch (all blocks resident), in two
// levels so that no counter takes more than GB_GROUP + gridDim.x / GB_GROUP
// arrivals: a block arrives at its group's count; the last of a group resets
// that count and arrives at the top count; the last group resets the top count
// and advances the generation.  Each counter has a 128-byte line of its own
// (word 0: top count, word 32: generation, word 64 + 32 g: group g), so the
// arrivals and the polls of the generation do not queue on one line.  The
// counts are zero at the first launch and left zero by every completed
// barrier.  The other blocks poll the generation at most `spin` times
// (sleeping briefly between polls) and give up after that, setting
// ST_TIMEOUT, so no wait is unbounded.  Returns false in every thread of a
// block that gave up (the counts are then stale: the host clears them before
// the next launch).  Grids of up to GBAR_MAX_BLOCKS blocks.
constexpr unsigned GB_GROUP = 16;

__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned spin, unsigned *status)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 32;
        const unsigned g = *gen;                     // read before arriving: it cannot move yet
        __threadfence();                             // this block's writes before its arrival
        const unsigned grp = blockIdx.x / GB_GROUP;
        const unsigned gsize = min(GB_GROUP, gridDim.x - grp * GB_GROUP);
        const unsigned ngroups = (gridDim.x + GB_GROUP - 1) / GB_GROUP;
        unsigned *gcount = bar + 64 + 32 * grp;
        int ok = 1;
        bool last = false;
        if (atomicAdd(gcount, 1u) == gsize - 1) {
            *gcount = 0u;
            __threadfence();
            if (atomicAdd(bar, 1u) == ngroups - 1) {
                bar[0] = 0u;
                last = true;
            }
        }
        if (last) {
            __threadfence();
            atomicAdd(bar + 32, 1u);
        } else {
            unsigned k = 0;
            while (*gen == g) {
                if (k++ >= spin) { ok = 0; atomicOr(status, (unsigned)ST_TIMEOUT); break; }
                if (k > 64) __nanosleep(64);             // busy first, then back off
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

}  // namespace fetdpic

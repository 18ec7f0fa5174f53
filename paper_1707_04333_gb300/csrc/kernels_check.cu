// Conservation checks of the FETD-PIC step (run every check_interval steps):
//   - nodal charge q_i = sum_p Q lambda_i(r_p) (Eq. (scatter.charge.assign)) in
//     the same 64-bit fixed point as the current, so the discrete continuity
//     residual (q^{n+1} - q^n)/dt + S~ i^{n+1/2} (Eq. (full.dis.cont)) is an
//     exact integer sum of rounding errors;
//   - discrete Gauss law S~ d^n - q^n against its initial value (Eq.
//     (semi.dis.div.2) in the dual-flux form d^{n+1} = d^n + dt (C^T H b - i));
//   - field energy e.[*eps].e/2 + b.[*mu^-1].b/2.
// Node sums gather over a node -> edge incidence list in a fixed order, and
// the energy uses a two-pass reduction, so every check value is deterministic.
#include <algorithm>

#include <cuda_runtime.h>

#include "fetdpic_internal.h"

namespace fetdpic {

// q_fix[node] += round(w lambda_i 2^shift): FP64 path from global coordinates.
__global__ void k_charge64(long long P, const int *__restrict__ cell, const short *__restrict__ blk_sp, int block,
                           const Species *__restrict__ sp, const Geo64 *__restrict__ geo,
                           const Topo *__restrict__ topo, const double *__restrict__ x,
                           const double *__restrict__ y, unsigned long long *__restrict__ q)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int f = cell[p];
    if (f < 0) return;
    const double w = sp[blk_sp[p / block]].qfix;
    const Geo64 &G = geo[f];
    const Topo &T = topo[f];
    const double px = x[p], py = y[p];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const int a = (m + 1) % 3;
        const double l = G.gx[m] * (px - G.X[a]) + G.gy[m] * (py - G.Y[a]);
        const long long v = __double2ll_rn(l * w);
        if (v) atomicAdd(q + T.node[m], (unsigned long long)v);
    }
}

// FP32 path: lambda = (l0, l1, 1 - l0 - l1) exactly as the particle kernel forms it.
__global__ void k_charge32(long long P, const int *__restrict__ cell, const short *__restrict__ blk_sp, int block,
                           const Species *__restrict__ sp, const Topo *__restrict__ topo,
                           const float *__restrict__ l0, const float *__restrict__ l1,
                           unsigned long long *__restrict__ q)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int f = cell[p];
    if (f < 0) return;
    const double w = sp[blk_sp[p / block]].qfix;
    const Topo &T = topo[f];
    const float a = l0[p], b = l1[p];
    const float c = 1.f - a - b;
    const float l[3] = {a, b, c};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const long long v = __double2ll_rn((double)l[m] * w);
        if (v) atomicAdd(q + T.node[m], (unsigned long long)v);
    }
}

__device__ __forceinline__ void atomic_max_pos(double *addr, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// Continuity residual per node: res = (q1 - q0) + sum_e o(k,e) i_e, exactly in
// integers; normalised by sum_e |i_e| + |q1 - q0| (at least one unit).
__global__ void k_dce(int N, const int *__restrict__ nrp, const int *__restrict__ nedge,
                      const int *__restrict__ ninst, const unsigned long long *__restrict__ ifix,
                      const unsigned long long *__restrict__ q0, const unsigned long long *__restrict__ q1,
                      double *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    long long flux = 0;
    double absf = 0.0;
    for (int r = nrp[k]; r < nrp[k + 1]; ++r) {
        const int w = nedge[r];
        const long long iv = (long long)ifix[w >> 1];
        flux += (w & 1) ? -iv : iv;
        absf += fabs((double)iv);
    }
    const long long dq = (long long)q1[k] - (long long)q0[k];
    const long long res = dq + flux;
    const double scale = fmax(absf + fabs((double)dq), 1.0);
    atomic_max_pos(out + 3 * ninst[k], fabs((double)res) / scale);
}

// Gauss residual per node: g = sum_e o(k,e) d_e - q (physical units).  With
// init != 0 it stores g as the reference g0; otherwise it reports
// |g - g0| / (sum |d_e| + |q| + |g0|).
__global__ void k_dgl(int N, const int *__restrict__ nrp, const int *__restrict__ nedge,
                      const int *__restrict__ ninst, const double *__restrict__ qunit,
                      const double *__restrict__ d, const unsigned long long *__restrict__ q,
                      double *__restrict__ g0, int init, double *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double s = 0.0, sa = 0.0;
    for (int r = nrp[k]; r < nrp[k + 1]; ++r) {
        const int w = nedge[r];
        const double v = d[w >> 1];
        s += (w & 1) ? -v : v;
        sa += fabs(v);
    }
    const int in = ninst[k];
    const double qk = (double)(long long)q[k] * qunit[in];
    const double g = s - qk;
    if (init) { g0[k] = g; return; }
    const double scale = sa + fabs(qk) + fabs(g0[k]);
    const double nr = scale > 0.0 ? fabs(g - g0[k]) / scale : 0.0;
    atomic_max_pos(out + 3 * in + 1, nr);
}

// Energy, first pass: per block, sum over its edges of e_k ([*eps] e)_k / 2 and
// over its faces of b_f^2 / (2 mu0 A_f), per instance; written to part[block].
__global__ void k_energy_part(int E, int F, const long long *__restrict__ hrp, const int *__restrict__ hci,
                              const double *__restrict__ hv, const double *__restrict__ e,
                              const int *__restrict__ einst, const double *__restrict__ b,
                              const Geo64 *__restrict__ geo, const Topo *__restrict__ topo,
                              int ninst, double *__restrict__ part)
{
    extern __shared__ double sh[];              // [blockDim.x]
    const int tid = threadIdx.x;
    const long long i = (long long)blockIdx.x * blockDim.x + tid;
    // one instance per block-level partial would need segmenting; keep it simple:
    // the partial of each block is per instance through a small loop
    for (int in = 0; in < ninst; ++in) {
        double v = 0.0;
        if (i < E && einst[i] == in) {
            double s = 0.0;
            for (long long q = hrp[i]; q < hrp[i + 1]; ++q) s += hv[q] * e[hci[q]];
            v += 0.5 * e[i] * s;
        }
        if (i < F && topo[i].inst == in) v += 0.5 * b[i] * b[i] * geo[i].hb;
        sh[tid] = v;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (tid < o) sh[tid] += sh[tid + o];
            __syncthreads();
        }
        if (tid == 0) part[(long long)blockIdx.x * ninst + in] = sh[0];
        __syncthreads();
    }
}

// Energy, second pass: one thread per instance sums the block partials in order.
__global__ void k_energy_final(long long nblocks, int ninst, const double *__restrict__ part, double *__restrict__ out)
{
    const int in = blockIdx.x * blockDim.x + threadIdx.x;
    if (in >= ninst) return;
    double s = 0.0;
    for (long long k = 0; k < nblocks; ++k) s += part[k * ninst + in];
    out[3 * in + 2] = s;
}

void launch_charge(cudaStream_t st, bool fp32, long long P, const int *cell, const short *blk_sp, int block,
                   const Species *sp, const Geo64 *geo, const Topo *topo, const void *f0, const void *f1,
                   unsigned long long *q, int N)
{
    cudaMemsetAsync(q, 0, sizeof(unsigned long long) * (size_t)N, st);
    if (P <= 0) return;
    const unsigned g = (unsigned)((P + 255) / 256);
    if (fp32) k_charge32<<<g, 256, 0, st>>>(P, cell, blk_sp, block, sp, topo, (const float *)f0, (const float *)f1, q);
    else k_charge64<<<g, 256, 0, st>>>(P, cell, blk_sp, block, sp, geo, topo, (const double *)f0, (const double *)f1, q);
}

void launch_dce(cudaStream_t st, int N, const int *nrp, const int *nedge, const int *ninst,
                const unsigned long long *ifix, const unsigned long long *q0, const unsigned long long *q1, double *out)
{
    if (N <= 0) return;
    k_dce<<<(N + 255) / 256, 256, 0, st>>>(N, nrp, nedge, ninst, ifix, q0, q1, out);
}

void launch_dgl(cudaStream_t st, int N, const int *nrp, const int *nedge, const int *ninst, const double *qunit,
                const double *d, const unsigned long long *q, double *g0, int init, double *out)
{
    if (N <= 0) return;
    k_dgl<<<(N + 255) / 256, 256, 0, st>>>(N, nrp, nedge, ninst, qunit, d, q, g0, init, out);
}

long long energy_blocks(int E, int F) { return ((long long)(E > F ? E : F) + 255) / 256; }

void launch_energy(cudaStream_t st, int E, int F, const long long *hrp, const int *hci, const double *hv,
                   const double *e, const int *einst, const double *b, const Geo64 *geo, const Topo *topo,
                   int ninst, double *part, double *out)
{
    const long long nb = energy_blocks(E, F);
    if (nb <= 0) return;
    k_energy_part<<<(unsigned)nb, 256, 256 * sizeof(double), st>>>(E, F, hrp, hci, hv, e, einst, b, geo, topo, ninst,
                                                                    part);
    k_energy_final<<<(ninst + 63) / 64, 64, 0, st>>>(nb, ninst, part, out);
}


// ------------------------------------------------------------- field probes
// One block: every thread reads the step counter before thread 0 advances it,
// so a captured graph writes consecutive ring rows on consecutive replays.
__global__ void __launch_bounds__(256) k_probe(long long n, const ProbeW *__restrict__ pw, const double *__restrict__ e,
                                               double2 *__restrict__ ring, long long cap,
                                               unsigned long long *count)
{
    const unsigned long long row = *count % (unsigned long long)cap;
    double2 *out = ring + (size_t)row * (size_t)n;
    for (long long p = threadIdx.x; p < n; p += blockDim.x) {
        const ProbeW w = pw[p];
        const double e0 = e[w.eg[0]], e1 = e[w.eg[1]], e2 = e[w.eg[2]];
        out[p] = make_double2(w.w[0] * e0 + w.w[2] * e1 + w.w[4] * e2, w.w[1] * e0 + w.w[3] * e1 + w.w[5] * e2);
    }
    __syncthreads();
    if (threadIdx.x == 0) *count += 1;
}

void launch_probe(cudaStream_t st, long long n, const ProbeW *pw, const double *e, double2 *ring, long long cap,
                  unsigned long long *count)
{
    if (n <= 0 || cap <= 0) return;
    k_probe<<<1, 256, 0, st>>>(n, pw, e, ring, cap, count);
}

}  // namespace fetdpic

// ------------------------------------------------- arithmetic-rate probe
// Measurement aid for the roofline of the arithmetic-bound FP64 particle path
// (no counterpart in the paper): eight independent FMA chains per thread,
// unrolled 16 deep, on a grid that fills every SM.
namespace fetdpic {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T seed, T *out)
{
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + (T)(threadIdx.x + k);
    const T m = (T)0.9999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == (T)-1) out[0] = s;                      // never true; keeps the chains live
}

}  // namespace fetdpic

extern "C" int fetdpic_fma_rate(int fp64, double *tflops)
{
    using namespace fetdpic;
    if (!tflops) return FETDPIC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FETDPIC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FETDPIC_ECUDA;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void *out = nullptr;
    int rc = FETDPIC_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMalloc(&out, 16) != cudaSuccess)
        rc = FETDPIC_ECUDA;
    const unsigned grid = (unsigned)sms * 8u;
    const double threads = (double)grid * 256.0;
    double best = 0.0;
    int iters = 64;
    for (int trial = 0; rc == FETDPIC_OK && trial < 12; ++trial) {
        cudaEventRecord(e0, st);
        if (fp64) k_fma_rate<double><<<grid, 256, 0, st>>>(iters, 1.0, (double *)out);
        else k_fma_rate<float><<<grid, 256, 0, st>>>(iters, 1.0f, (float *)out);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = FETDPIC_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < 20.f) { iters = (int)std::min(1 << 22, iters * 2); continue; }   // grow to >= 20 ms
        best = std::max(best, 2.0 * 8 * 16 * (double)iters * threads / (ms * 1e-3) / 1e12);
    }
    if (rc == FETDPIC_OK && cudaGetLastError() != cudaSuccess) rc = FETDPIC_ECUDA;
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    *tflops = best;
    return rc;
}

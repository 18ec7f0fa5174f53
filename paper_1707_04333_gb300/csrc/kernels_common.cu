// Field-update (Ampere) kernels, the counting sort of particles by triangle,
// the scan it needs, and the kernels that return particles in load order.
#include <algorithm>
#include <type_traits>

#include <cuda_runtime.h>

#include "fetdpic_internal.h"
#include "field_device.cuh"

namespace fetdpic {

// e_free += (dt M) r for one row: SpMV with the dt-scaled SPAI in sliced ELL
// (slices of 32 rows, each padded to its longest row and stored column-major,
// so a warp of consecutive rows reads 32 consecutive column indices and values
// per step).  Padding entries have value 0 and a valid column.  r is read
// through the coherent path: the fused kernel writes it earlier in the launch.
template <typename V>
__device__ __forceinline__ void spai_row(const AmpereArgs &a, const V *__restrict__ v, const V *r,
                                         long long row, unsigned long long keep)
{
    const long long sl = row >> 5;
    const int lane = (int)(row & 31);
    const long long o0 = a.m_soff[sl], o1 = a.m_soff[sl + 1];
    V s0 = V(0), s1 = V(0);
    long long q = o0 + lane;
    for (; q + 32 < o1; q += 64) {
        s0 += ld_keep(v + q, keep) * r[ld_keep(a.m_ci + q, keep)];
        s1 += ld_keep(v + q + 32, keep) * r[ld_keep(a.m_ci + q + 32, keep)];
    }
    if (q < o1) s0 += ld_keep(v + q, keep) * r[ld_keep(a.m_ci + q, keep)];
    a.e[a.m_row[row]] += (double)(s0 + s1);
}

// The same row behind the wait for the kernel that writes r: before the wait
// only the lines of its first two entries (values and columns, static) are
// pulled into L1, so their latency overlaps that kernel's end while the row is
// summed by spai_row itself (same loop, same order: the result is the same).
// (Loading those entries into registers before the wait and entering the loop
// after them gave the same on the 200k-triangle mesh but made the
// bandwidth-bound SpMV of the 64-instance batch 13 % slower.)
template <typename V>
__device__ __forceinline__ void spai_row_pdl(const AmpereArgs &a, const V *__restrict__ v, const V *r,
                                             long long row, unsigned long long keep)
{
    const long long sl = row >> 5;
    const int lane = (int)(row & 31);
    const long long o0 = a.m_soff[sl], o1 = a.m_soff[sl + 1];
    const long long q = o0 + lane;
    if (q < o1) {
        asm volatile("prefetch.global.L1 [%0];" ::"l"(v + q));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.m_ci + q));
    }
    if (q + 32 < o1) {
        asm volatile("prefetch.global.L1 [%0];" ::"l"(v + q + 32));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.m_ci + q + 32));
    }
    pdl_begin();
    spai_row<V>(a, v, r, row, keep);
}

// Matrices up to this size are prefetched before the wait (they stay in the
// 129 MB L2 between steps, loaded with an evict-last policy).
constexpr long long SPMV_PREFETCH_MAX_BYTES = 64ll << 20;

// (Loading the face pairs and coefficients before the wait, as the SpMV does with
// its operands, measured slower on GB300: 23.1 -> 26.5 us per step for the curl
// and the SpMV together with stage events.)
__global__ void k_curl_h(AmpereArgs a)
{
    pdl_begin();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.E) return;
    curl_h_edge(a, e, l2_keep());
}

// PRE: prefetch before the wait (a matrix that stays in L2: the SpMV is bound
// by latency); else wait first (a large matrix: bound by HBM bandwidth, where
// the prefetches only add requests).
template <typename V, bool PRE>
__global__ void __launch_bounds__(256) k_spai_sell(AmpereArgs a)
{
    const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!PRE) pdl_begin();
    if (row >= a.nfree) { if (PRE) pdl_begin(); return; }
    if constexpr (PRE) {
        if constexpr (sizeof(V) == 4) spai_row_pdl<float>(a, a.m_v32, a.r32, row, l2_keep());
        else spai_row_pdl<double>(a, a.m_v, a.r, row, l2_keep());
    } else {
        if constexpr (sizeof(V) == 4) spai_row<float>(a, a.m_v32, a.r32, row, l2_keep());
        else spai_row<double>(a, a.m_v, a.r, row, l2_keep());
    }
}


// Both Ampere phases in one cooperative launch: r on every edge (grid-stride),
// a grid barrier (the SpMV reads r anywhere), then e += dt M r on every free
// row (grid-stride; a warp takes 32 consecutive rows, one slice).  Same
// per-edge and per-row arithmetic as the two separate kernels, so the result
// is bit-identical to them.
constexpr int FUSED_BLOCK = 1024;              // one block per SM: few arrivals at the barrier

template <typename V>
__global__ void __launch_bounds__(FUSED_BLOCK) k_ampere_fused(AmpereArgs a)
{
    const unsigned long long keep = l2_keep();
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long e = tid; e < a.E; e += nth) curl_h_edge(a, (int)e, keep);
    if (!grid_barrier(a.gbar, a.spin, a.status)) return;
    for (long long row = tid; row < a.nfree; row += nth) {
        if constexpr (sizeof(V) == 4) spai_row<float>(a, a.m_v32, a.r32, row, keep);
        else spai_row<double>(a, a.m_v, a.r, row, keep);
    }
}

template <typename V>
static void launch_fused(cudaStream_t st, const AmpereArgs &a)
{
    static int per_sm = 0, sms = 0, dev = -1;
    int d = 0;
    cudaGetDevice(&d);
    if (d != dev || per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ampere_fused<V>, FUSED_BLOCK, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        dev = d;
        if (per_sm < 1) per_sm = 1;
    }
    const long long work = std::max<long long>(a.E, a.nfree);
    const long long grid = std::min<long long>(std::min<long long>((work + FUSED_BLOCK - 1) / FUSED_BLOCK,
                                                                    (long long)per_sm * sms),
                                                GBAR_MAX_BLOCKS);
    AmpereArgs arg = a;
    void *params[] = {&arg};
    cudaLaunchCooperativeKernel((const void *)k_ampere_fused<V>, dim3((unsigned)grid), dim3(FUSED_BLOCK), params, 0,
                                st);
}

void launch_ampere(cudaStream_t st, const AmpereArgs &a)
{
    if (a.E <= 0 && a.nfree <= 0) return;
    if (a.fused) {
        if (a.m_v32) launch_fused<float>(st, a);
        else launch_fused<double>(st, a);
        return;
    }
    if (a.E > 0) launch_k(a.pdl, k_curl_h, dim3((a.E + 255) / 256), dim3(256), st, a);
    if (a.nfree > 0) {
        const dim3 g((unsigned)((a.nfree + 255) / 256));
        // matrix bytes (values and columns, padding included) against what stays in L2
        const long long bytes = a.m_entries * (long long)((a.m_v32 ? 4 : 8) + 4);
        const bool pre = bytes <= SPMV_PREFETCH_MAX_BYTES;
        if (a.m_v32) {
            if (pre) launch_k(a.pdl, k_spai_sell<float, true>, g, dim3(256), st, a);
            else launch_k(a.pdl, k_spai_sell<float, false>, g, dim3(256), st, a);
        } else {
            if (pre) launch_k(a.pdl, k_spai_sell<double, true>, g, dim3(256), st, a);
            else launch_k(a.pdl, k_spai_sell<double, false>, g, dim3(256), st, a);
        }
    }
}

// ------------------------------------------------------------------- scan
// Exclusive scan of n ints: per-block totals, then block scans offset by the
// totals of the blocks before them.

constexpr int SCAN_B = 1024;

__device__ __forceinline__ int block_exclusive_scan(int v, int *sh, int &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const int before = (w > 0 ? sh[w - 1] : 0) + x - v;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_scan_sums(const int *__restrict__ in, long long n, int *__restrict__ sums)
{
    __shared__ int sh[32];
    const long long i = (long long)blockIdx.x * SCAN_B + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    int tot;
    block_exclusive_scan(v, sh, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Block b adds the sum of the block totals before it (a block reduction over
// at most n / 1024 totals) to its own exclusive scan.
__global__ void k_scan_apply(const int *__restrict__ in, long long n, const int *__restrict__ sums, int *__restrict__ out)
{
    __shared__ int sh[32];
    int pre = 0;
    for (long long k = threadIdx.x; k < (long long)blockIdx.x; k += SCAN_B) pre += sums[k];
    pre = __reduce_add_sync(0xffffffffu, pre);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = pre;
    __syncthreads();
    int carry = 0;
#pragma unroll 1
    for (int k = 0; k < SCAN_B / 32; ++k) carry += sh[k];
    __syncthreads();
    const long long i = (long long)blockIdx.x * SCAN_B + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    int tot;
    const int ex = block_exclusive_scan(v, sh, tot);
    if (i < n) out[i] = ex + carry;
}

size_t scan_tmp_ints(long long n) { return (size_t)((n + SCAN_B - 1) / SCAN_B) + 1; }

void launch_exclusive_scan(cudaStream_t st, const int *in, int *out, long long n, int *tmp)
{
    if (n <= 0) return;
    const long long nb = (n + SCAN_B - 1) / SCAN_B;
    k_scan_sums<<<(unsigned)nb, SCAN_B, 0, st>>>(in, n, tmp);
    k_scan_apply<<<(unsigned)nb, SCAN_B, 0, st>>>(in, n, tmp, out);
}

// ------------------------------------------------------------------- sort
// Counting sort by triangle within each species range: histogram (integer
// atomics), exclusive scan, scatter through per-triangle cursors.  The bins of
// species s are its triangles, then one bin for its padding slots (and the
// slots of particles dropped by a write), so the bins of a species count its
// whole storage range: the scan gives storage slots directly, every slot of
// the output is written once, and a species whose live count fell keeps its
// range.  The order
// of particles inside one triangle depends on atomic order; nothing computed
// depends on it (the deposit is integer, reads go through the id array).

// Runs of equal key among the lanes of a warp (adjacent lanes only: the
// particles are nearly sorted, so runs are long; a key that comes back later
// in the warp starts a run of its own).  head: first lane of its run; lead:
// that run's first lane; len: the run's length (valid on its first lane).
struct WarpRun { bool head; int lead, len; };
__device__ __forceinline__ WarpRun warp_run(int key, int lane)
{
    const unsigned full = 0xffffffffu;
    const int kn = __shfl_down_sync(full, key, 1);
    const int kp = __shfl_up_sync(full, key, 1);
    const unsigned tails = __ballot_sync(full, lane == 31 || kn != key);
    const bool head = lane == 0 || kp != key;
    const unsigned heads = __ballot_sync(full, head);
    WarpRun r;
    r.head = head;
    r.lead = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    r.len = __ffs(tails >> lane);
    return r;
}

// Bin of a slot of a species: its triangle, or the padding bin after them.
__device__ __forceinline__ int sort_bin(int c, int hoff, const Species &s)
{
    return c < 0 ? hoff + s.nf : hoff + (c - s.cell_off);
}

// Histogram: one integer atomic per run of equal triangle in a warp.  Each
// warp takes HI_UNROLL consecutive 32-particle chunks at a time, their keys
// loaded before any is used, so several loads per warp are in flight; the grid
// is one wave, striding over the chunks.
constexpr int HI_UNROLL = 8;

__global__ void __launch_bounds__(256) k_hist(long long nchunks, const int *__restrict__ cell,
                                              const short *__restrict__ chunk_sp, const Species *__restrict__ sp,
                                              const int *__restrict__ hoff, int *__restrict__ hist)
{
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c0 = w * HI_UNROLL; c0 < nchunks; c0 += nw * HI_UNROLL) {
        int cc[HI_UNROLL], sid[HI_UNROLL];
#pragma unroll
        for (int k = 0; k < HI_UNROLL; ++k) {
            const long long ch = c0 + k;
            cc[k] = -1; sid[k] = -1;
            if (ch < nchunks) { cc[k] = __ldcs(cell + ch * 32 + lane); sid[k] = chunk_sp[ch]; }
        }
#pragma unroll
        for (int k = 0; k < HI_UNROLL; ++k) {
            const int slot = sid[k] < 0 ? -1 : sort_bin(cc[k], hoff[sid[k]], sp[sid[k]]);
            const WarpRun r = warp_run(slot, lane);
            if (slot >= 0 && r.head) atomicAdd(hist + slot, r.len);
        }
    }
}

// Scatter through per-triangle cursors.  Each warp handles SC_CHUNKS
// consecutive 32-particle chunks: all cursor atomics are issued before any of
// their results is used, then the payload moves.
constexpr int SC_CHUNKS = 4;

template <int FB>
__global__ void __launch_bounds__(256) k_scatter(long long nchunks, const int *__restrict__ cell,
                                                 const int *__restrict__ id, const short *__restrict__ chunk_sp,
                                                 const Species *__restrict__ sp, const int *__restrict__ hoff,
                                                 int *__restrict__ cursor,
                                                 const void *f0, const void *f1, const void *f2, const void *f3,
                                                 int *__restrict__ cell_o, int *__restrict__ id_o,
                                                 void *g0, void *g1, void *g2, void *g3)
{
    using T = typename std::conditional<FB == 8, double, float>::type;
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long c0 = w * SC_CHUNKS;
    int cc[SC_CHUNKS], slot[SC_CHUNKS], sid[SC_CHUNKS], base[SC_CHUNKS], rank[SC_CHUNKS];
    unsigned peers[SC_CHUNKS];
    // the payload is loaded with the keys, so its DRAM latency overlaps the cursor atomics
    int idv[SC_CHUNKS];
    T v0[SC_CHUNKS], v1[SC_CHUNKS], v2[SC_CHUNKS], v3[SC_CHUNKS];
#pragma unroll
    for (int k = 0; k < SC_CHUNKS; ++k) {
        const long long ch = c0 + k;
        cc[k] = -1; sid[k] = -1;
        if (ch < nchunks) {
            const long long p = ch * 32 + lane;
            cc[k] = cell[p]; sid[k] = chunk_sp[ch];
            idv[k] = id[p];
            v0[k] = ((const T *)f0)[p]; v1[k] = ((const T *)f1)[p];
            v2[k] = ((const T *)f2)[p]; v3[k] = ((const T *)f3)[p];
        }
    }
#pragma unroll
    for (int k = 0; k < SC_CHUNKS; ++k) {
        slot[k] = sid[k] < 0 ? -1 : sort_bin(cc[k], hoff[sid[k]], sp[sid[k]]);
        peers[k] = __match_any_sync(0xffffffffu, slot[k]);
        rank[k] = __popc(peers[k] & ((1u << lane) - 1u));
        base[k] = 0;
        if (slot[k] >= 0 && lane == __ffs(peers[k]) - 1) base[k] = atomicAdd(cursor + slot[k], __popc(peers[k]));
    }
#pragma unroll
    for (int k = 0; k < SC_CHUNKS; ++k) {
        const int leader = __ffs(peers[k]) - 1;
        const int b = __shfl_sync(0xffffffffu, base[k], leader);
        if (slot[k] < 0) continue;
        const long long q = (long long)(b + rank[k]);
        cell_o[q] = cc[k];
        id_o[q] = idv[k];
        ((T *)g0)[q] = v0[k];
        ((T *)g1)[q] = v1[k];
        ((T *)g2)[q] = v2[k];
        ((T *)g3)[q] = v3[k];
    }
}

// SM count of the current device (cached per device).
static int sort_sms()
{
    static int sms = 0, dev = -1;
    int d = 0;
    cudaGetDevice(&d);
    if (d != dev || sms == 0) { cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d); dev = d; }
    return sms;
}

void launch_sort(cudaStream_t st, const SortArgs &a)
{
    cudaMemsetAsync(a.hist, 0, sizeof(int) * a.hist_n, st);
    {
        const long long nch = a.P / 32;
        const long long need = (nch + 8 * HI_UNROLL - 1) / (8 * HI_UNROLL);    // 8 warps per block
        const long long grid = std::max<long long>(1, std::min<long long>(need, 8LL * sort_sms()));
        k_hist<<<(unsigned)grid, 256, 0, st>>>(nch, a.cell, a.chunk_sp, a.sp_dev, a.hoff, a.hist);
    }
    // exclusive scan in place into the cursor array (hist doubles as cursor)
    launch_exclusive_scan(st, a.hist, a.hist, a.hist_n, a.scan_tmp);
    const long long nchunks = a.P / 32;
    const long long warps = (nchunks + SC_CHUNKS - 1) / SC_CHUNKS;
    const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    if (a.fbytes == 8)
        k_scatter<8><<<grid, 256, 0, st>>>(nchunks, a.cell, a.id, a.chunk_sp, a.sp_dev, a.hoff, a.hist,
                                           a.f[0], a.f[1], a.f[2], a.f[3], a.cell_tmp, a.id_tmp, a.f_tmp[0],
                                           a.f_tmp[1], a.f_tmp[2], a.f_tmp[3]);
    else
        k_scatter<4><<<grid, 256, 0, st>>>(nchunks, a.cell, a.id, a.chunk_sp, a.sp_dev, a.hoff, a.hist,
                                           a.f[0], a.f[1], a.f[2], a.f[3], a.cell_tmp, a.id_tmp, a.f_tmp[0],
                                           a.f_tmp[1], a.f_tmp[2], a.f_tmp[3]);
}

// ------------------------------------------------------------ load order

// Host-layout particle state (x, u in FP64, instance-local cell) into the
// storage range of one species, in load order.  FP32 storage gets the
// barycentric coordinates of x in its triangle and u/c.
// An instance-local triangle outside [0, nf) is never used as an address: the
// particle becomes padding and ST_BADCELL reports it at the next sync.
__global__ void k_ingest(long long n, long long cap, long long off, int cell_off, int nf, int fp32, const double *__restrict__ x,
                         const double *__restrict__ u, const int *__restrict__ cell, const int *__restrict__ c2i,
                         const Geo64 *__restrict__ geo, double inv_c, int *__restrict__ cell_o,
                         int *__restrict__ id_o, void *f0, void *f1, void *f2, void *f3, unsigned *status)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cap) return;
    const long long p = off + k;
    if (k >= n) {                          // the species' padding: no particle, no load index
        cell_o[p] = -1;
        id_o[p] = -1;
        return;
    }
    const int cl = cell[k];
    if (cl < 0 || cl >= nf) {
        cell_o[p] = -1;
        id_o[p] = (int)k;
        atomicOr(status, (unsigned)ST_BADCELL);
        return;
    }
    const int c = cell_off + c2i[cell_off + cl];
    cell_o[p] = c;
    id_o[p] = (int)k;
    const double px = x[2 * k], py = x[2 * k + 1];
    if (fp32) {
        const Geo64 &G = geo[c];
        const double l0 = G.gx[0] * (px - G.X[1]) + G.gy[0] * (py - G.Y[1]);
        const double l1 = G.gx[1] * (px - G.X[2]) + G.gy[1] * (py - G.Y[2]);
        ((float *)f0)[p] = (float)l0;
        ((float *)f1)[p] = (float)l1;
        ((float *)f2)[p] = (float)(u[2 * k] * inv_c);
        ((float *)f3)[p] = (float)(u[2 * k + 1] * inv_c);
    } else {
        ((double *)f0)[p] = px;
        ((double *)f1)[p] = py;
        ((double *)f2)[p] = u[2 * k];
        ((double *)f3)[p] = u[2 * k + 1];
    }
}

void launch_ingest(cudaStream_t st, long long n, long long cap, long long off, int cell_off, int nf, bool fp32,
                   const double *x, const double *u, const int *cell, const int *c2i, const Geo64 *geo,
                   double inv_c, int *cell_o, int *id_o, void *f0, void *f1, void *f2, void *f3, unsigned *status)
{
    if (cap <= 0) return;
    k_ingest<<<(unsigned)((cap + 255) / 256), 256, 0, st>>>(n, cap, off, cell_off, nf, fp32 ? 1 : 0, x, u, cell, c2i,
                                                            geo, inv_c, cell_o, id_o, f0, f1, f2, f3, status);
}

__global__ void k_unsort64(long long off, long long cap, long long n, const int *__restrict__ cell, const int *__restrict__ id,
                           const double *__restrict__ x, const double *__restrict__ y,
                           const double *__restrict__ ux, const double *__restrict__ uy, const int *__restrict__ i2c,
                           double *__restrict__ ox, double *__restrict__ ou, int *__restrict__ oc)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cap) return;
    const long long p = off + k;
    const int c = cell[p];
    const long long i = id[p];
    if (c < 0) {
        // a particle dropped by a write keeps its load index: it reads NaN and triangle -1
        if (i >= 0 && i < n) {
            if (ox) { ox[2 * i] = __longlong_as_double(-1ll); ox[2 * i + 1] = __longlong_as_double(-1ll); }
            if (ou) { ou[2 * i] = __longlong_as_double(-1ll); ou[2 * i + 1] = __longlong_as_double(-1ll); }
            if (oc) oc[i] = -1;
        }
        return;
    }
    if (ox) { ox[2 * i] = x[p]; ox[2 * i + 1] = y[p]; }
    if (ou) { ou[2 * i] = ux[p]; ou[2 * i + 1] = uy[p]; }
    if (oc) oc[i] = i2c[c];
}

__global__ void k_unsort32(long long off, long long cap, long long n, const int *__restrict__ cell, const int *__restrict__ id,
                           const float *__restrict__ l0, const float *__restrict__ l1,
                           const float *__restrict__ ux, const float *__restrict__ uy,
                           const Geo64 *__restrict__ geo, double c, const int *__restrict__ i2c,
                           double *__restrict__ ox, double *__restrict__ ou, int *__restrict__ oc)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cap) return;
    const long long p = off + k;
    const int f = cell[p];
    const long long i = id[p];
    if (f < 0) {
        // a particle dropped by a write keeps its load index: it reads NaN and triangle -1
        if (i >= 0 && i < n) {
            if (ox) { ox[2 * i] = __longlong_as_double(-1ll); ox[2 * i + 1] = __longlong_as_double(-1ll); }
            if (ou) { ou[2 * i] = __longlong_as_double(-1ll); ou[2 * i + 1] = __longlong_as_double(-1ll); }
            if (oc) oc[i] = -1;
        }
        return;
    }
    if (ox) {
        const double a = l0[p], b = l1[p];
        const double cc = 1.0 - a - b;
        const Geo64 &G = geo[f];
        ox[2 * i] = a * G.X[0] + b * G.X[1] + cc * G.X[2];
        ox[2 * i + 1] = a * G.Y[0] + b * G.Y[1] + cc * G.Y[2];
    }
    if (ou) { ou[2 * i] = (double)ux[p] * c; ou[2 * i + 1] = (double)uy[p] * c; }
    if (oc) oc[i] = i2c[f];
}

void launch_unsort64(cudaStream_t st, long long n, const int *cell, const int *id, const double *x,
                     const double *y, const double *ux, const double *uy, long long off, long long cap,
                     const int *i2c, double *ox, double *ou, int *oc)
{
    if (cap <= 0) return;
    k_unsort64<<<(unsigned)((cap + 255) / 256), 256, 0, st>>>(off, cap, n, cell, id, x, y, ux, uy, i2c, ox, ou, oc);
}

void launch_unsort32(cudaStream_t st, long long n, const int *cell, const int *id, const float *l0,
                     const float *l1, const float *ux, const float *uy, const Geo64 *geo, double c,
                     long long off, long long cap, const int *i2c, double *ox, double *ou, int *oc)
{
    if (cap <= 0) return;
    k_unsort32<<<(unsigned)((cap + 255) / 256), 256, 0, st>>>(off, cap, n, cell, id, l0, l1, ux, uy, geo, c, i2c,
                                                              ox, ou, oc);
}


}  // namespace fetdpic

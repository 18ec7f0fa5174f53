// Internal declarations of the fetdpic library (host setup, device records,
// kernel launchers).  Not part of the public C ABI (include/fetdpic.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fetdpic.h"

namespace fetdpic {

// ------------------------------------------------------------ host setup

// One mesh instance after validation: counter-clockwise triangles, edge
// numbering, incidence (Sec. II.A), Whitney geometry and matrices.
struct HostMesh {
    int nn = 0, nf = 0, ne = 0;
    std::vector<double> xy;                 // [nn][2]
    std::vector<int> tri;                   // [nf][3] CCW
    std::vector<int> edge;                  // [ne][2] orientation i -> j
    std::vector<int> tedge, tsign;          // [nf][3] edge of local edge m, +-1
    std::vector<int> tnb, tnbm;             // [nf][3] neighbour triangle / its local edge index, -1 at walls
    std::vector<char> pec;                  // [ne] e held at 0
    std::vector<int> efac;                  // [ne][2] adjacent triangles (second = -1 on walls)
    std::vector<int> efsign;                // [ne][2] circulation sign of the edge in each triangle
    std::vector<double> d2A, inv2A;         // [nf]
    std::vector<double> gx, gy, X, Y;       // [nf][3] grad lambda_m, node coordinates
    // periodic walls: node n is the same node as rep[n]; crossing local edge m of
    // triangle f moves a position by tshift[3f+m] * (tx, ty)
    bool periodic = false;
    std::vector<int> rep;                   // [nn]
    std::vector<signed char> tshift;        // [nf][3] in {-1, 0, 1}
    double tx = 0.0, ty = 0.0;
    std::vector<double> evec;               // [ne][2] r_j - r_i read off a triangle holding the edge
    // [*eps] restricted to free edges, CSR over free-edge indices
    std::vector<int> free_edges;            // ascending edge ids
    std::vector<long long> a_rp; std::vector<int> a_ci; std::vector<double> a_v;
    // full [*eps] over all edges (for d^0 = [*eps] e^0 and the field energy)
    std::vector<long long> h_rp; std::vector<int> h_ci; std::vector<double> h_v;
    // SPAI M ~ [*eps]^-1, CSR with free-edge rows and edge-id columns
    std::vector<long long> m_rp; std::vector<int> m_ci; std::vector<double> m_v;
    // triangle order: the library stores triangles along a Hilbert curve of their centroids;
    // perm[internal] = the caller's index, inv[caller] = internal index
    std::vector<int> perm, inv;
};

// Order of the triangles along a Hilbert curve of their centroids (ties by
// index): perm[k] = the caller's index of the k-th triangle.  Neighbours end up
// close in memory, so particles that have crossed into a neighbour since the
// last sort, and the sort's scattered writes, stay within cached lines.
std::vector<int> hilbert_order(int nn, const double *xy, int nf, const int *tri);

// Returns 0 or a negative fetdpic_status; msg gets a reason on error.
// tri: triangles in the caller's order; they are stored in hilbert_order.
int build_mesh(HostMesh &M, int nn, const double *xy, int nf, const int *tri,
               int ne_in, const int *edges_in, const int *tags_in,
               int n_per, const int *per_nodes, double tx, double ty, std::string &msg);
int build_hodge(HostMesh &M, double eps0, std::string &msg);
int build_spai(HostMesh &M, int level, std::string &msg);

// Initial electrostatic field of nodal charges q [nn] (node ids of the mesh;
// images of periodic nodes carry none): solves G^T [*eps] G phi = q on the
// nodes off the PEC walls (phi = 0 on them) by Jacobi-preconditioned
// conjugate gradients and returns de = -G phi [ne] (0 on PEC edges).
int electrostatic_solve(const HostMesh &M, const std::vector<double> &q, std::vector<double> &de,
                        int &iterations, double &rel_residual, std::string &msg);

// Same barycentric evaluation the kernels use (gradient form, no FMA).
void host_lambdas(const HostMesh &M, int f, double x, double y, double *l);
int host_locate(const HostMesh &M, double x, double y, int hint);

// --------------------------------------------------------- device records

// FP64 geometry of one triangle: lambda_m(r) = gx_m (x - X_{m+1}) + gy_m (y - Y_{m+1}).
struct __align__(16) Geo64 {
    double gx[3], gy[3], X[3], Y[3];
    double inv2A, dt, hb, pad;              // hb = 1/(mu0 A): diagonal [*mu^-1]
};
static_assert(sizeof(Geo64) == 128, "Geo64 layout");

// FP32 per-triangle constants, split by who reads them.  CstA (32 B, one
// 256-bit load): G_m = c dt grad lambda_m for m = 0, 1 (barycentric step per
// unit v/c; G_2 = -(G_0 + G_1) because the gradients sum to zero), edge words
// 1 and 2, neighbour words 0 and 1.  CstB (8 B): edge word 0 and neighbour
// word 2, read by the walk (the particle pass gets edge word 0 from the field
// record, where the Faraday kernel copies it).  Edge and neighbour words as in
// Topo.
struct __align__(32) CstA {
    float G[4];                             // (G0x, G0y, G1x, G1y)
    int ew1, ew2;
    int nb0, nb1;
};
static_assert(sizeof(CstA) == 32, "CstA layout");
struct __align__(8) CstB { int ew0, nb2; };
static_assert(sizeof(CstB) == 8, "CstB layout");

// FP32-path species parameters (32 B): q/m and the fixed-point weight first,
// read by the particle pass in one 8-byte uniform load.  Applied fields reach
// the FP32 path through the per-triangle field record, not through here.
struct __align__(16) Sp32 {
    float kappa;                            // q/m
    float wfix;                             // (q / q_ref) * (2^25 - 64)
    int inst, edge_off;
    int off;                                // storage offset of the species (walk record index base)
    int pad[3];
};
static_assert(sizeof(Sp32) == 32, "Sp32 layout");

// Topology: edge word = (global edge << 1) | (sign < 0); neighbour word =
// (global triangle << 2) | local index of the shared edge there, -1 on a wall.
struct __align__(16) Topo {
    int ew[3];
    int nb[3];
    int node[3];
    int inst;
};
static_assert(sizeof(Topo) == 48, "Topo layout");

// Fields seen by the particles of one triangle at step n (written by the
// Faraday kernel): FP64 path: (s_m e_m for m = 0..2, B_z^n); FP32 path:
// E(lambda) = sum_n lambda_n V_n scaled by dt/(2c), B_z scaled by dt/2.
struct __align__(32) Rec64 { double se[3]; double bz; };
struct __align__(32) Rec32 { float v[6]; float bz; int ew0; };

struct Species {
    double alpha;                           // q dt / (2 m)
    double wfix;                            // (q / q_ref) * 2^shift: deposit weight in fixed point
    double qfix;                            // same for the nodal charge
    double dt, c, ic2;
    double ext_ex, ext_ey, ext_bz;
    float kappa;                            // q/m (FP32 path)
    float xe_x, xe_y, xb;                   // external fields pre-scaled for the FP32 path
    float wfix32;
    int inst;
    int pad_;
    long long off, n, cap;                  // storage range [off, off+cap), n live
    int cell_off, nf;                       // triangle range of the instance
};

// Grid-barrier state: a top count, a generation and one count per 16 blocks,
// each on a 128-byte line of its own; enough for cooperative grids of up to
// GBAR_MAX_BLOCKS blocks.
constexpr int GBAR_MAX_BLOCKS = 4096;
constexpr int GBAR_WORDS = 64 + 32 * (GBAR_MAX_BLOCKS / 16);

enum StatusBits : unsigned {
    ST_WALK = 1u, ST_NONFINITE = 2u, ST_MESH = 4u, ST_TIMEOUT = 8u,
    ST_BADCELL = 16u                        // a written particle named a triangle outside its mesh
};

// ----------------------------------------------------------- launchers
// All launchers enqueue on `st` and return immediately.

#ifdef __CUDACC__
// Programmatic dependent launch: with pdl set, the kernel may be launched
// while the kernel before it on the stream still runs (its blocks become
// resident as room frees up), which hides the launch gap between the stages of
// a step.  Every kernel launched this way starts with pdl_begin(), whose
// griddepcontrol.wait returns only when the previous kernel has completed and
// its memory is visible; it then lets the next kernel launch early in turn.
// Without pdl this is a plain launch (and the wait returns at once).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

struct StepArgs64 {
    const Geo64 *geo; const Topo *topo; const Rec64 *rec;
    const Species *sp; const short *blk_sp;
    double *x, *y, *ux, *uy; int *cell;
    unsigned long long *ifix;               // [E] fixed-point current (two's complement)
    unsigned *status;
    int max_cross;
    int rec_cap; int *rec_cnt; int *wrec;   // walk record (rec_cap = 0: off), indexed by
                                            // species storage offset + load index, so a sort
                                            // after the step does not move it
    const int *id;                          // load index of each particle slot
    const int *edge_off;                    // per instance, for instance-local record ids
    long long nblocks; int block;
    const signed char *tshift;              // [F][3] periodic shift codes; NULL = no periodic walls
    const double2 *period;                  // per instance (tx, ty)
    const double2 *extw;                    // [F] weights (E, B) of the applied fields; NULL = 1
    const double *ext_amp;                  // per instance: amplitude of the applied E
};

struct StepArgs32 {
    const CstA *csta; const CstB *cstb; const Rec32 *rec;
    const Sp32 *sp; const short *chunk_sp;  // species of each 32-particle chunk
    long long nchunks;
    int variant;                            // particle-kernel variant (min resident blocks per SM)
    bool pdl;                               // programmatic dependent launch (launch_k)
    float *l0, *l1, *ux, *uy; int *cell;
    unsigned long long *ifix;
    unsigned *status;
    int max_cross;
    int rec_cap; int *rec_cnt; int *wrec;   // walk record, indexed as in StepArgs64
    const int *id;
    const int *edge_off;
    long long nblocks; int block;
    unsigned spin;                          // polls of a bounded wait before it gives up (variant 5)
};

void launch_faraday64(cudaStream_t st, int F, const Geo64 *geo, const Topo *topo, const double *e,
                      double *b, Rec64 *rec);
// Applied fields folded into the FP32 field record (ext == NULL: none): per
// instance (E_x, E_y, B_z, 0) times the amplitude (E) and the per-triangle
// weights extw (NULL = 1); finst = instance of each triangle.
struct __align__(16) ExtField { double ex, ey, bz, pad; };
struct Ext32 { const int *finst; const ExtField *ext; const double *amp; const double2 *extw; double half_over_c; };
void launch_faraday32(cudaStream_t st, int F, const CstA *csta, const CstB *cstb, const double2 *dtinv, const double *e,
                      double *b, Rec32 *rec, float inv2c2, const Ext32 &x, bool pdl);
void launch_particles64(cudaStream_t st, int pusher, const StepArgs64 &a);
void launch_particles32(cudaStream_t st, int pusher, const StepArgs32 &a);

struct AmpereArgs {
    int E;
    const int2 *efac; const double2 *ecoef;  // adjacent triangles, s_f / (mu0 A_f)
    const int *einst;                         // instance of each edge
    const double *inst_unit;                  // (q_ref/dt) 2^-shift per instance
    const double *inst_dt;
    const double *b;
    unsigned long long *ifix;                 // read and cleared
    double *r, *d, *j;
    float *r32;                               // FP32 copy of r (FP32 path), or null
    long long nfree;
    // dt-scaled SPAI in sliced ELL: slice offsets, row -> edge, columns, values (FP64 or FP32)
    const long long *m_soff; const int *m_row; const int *m_ci; const double *m_v; const float *m_v32;
    long long m_entries;                      // stored entries (padding included)
    double *e;
    // one cooperative launch for both phases (fused = true): its grid barrier's state (zero at
    // creation, left zero by every completed barrier, cleared by the host after a timeout), the
    // polls of its bounded wait, and the status word a wait that gives up sets
    bool fused;
    bool pdl;                                 // programmatic dependent launch (two-launch form)
    unsigned *gbar;
    unsigned spin;
    unsigned *status;
};
void launch_ampere(cudaStream_t st, const AmpereArgs &a);

// Counting sort of particles by triangle, per species range.
struct SortArgs {
    int nsp; const Species *sp_dev; const Species *sp_host;
    long long P;                              // storage size (padded)
    int *cell; int *cell_tmp;
    int *id; int *id_tmp;
    void *f[4]; void *f_tmp[4]; int fbytes;   // four payload arrays of fbytes each
    int *hist;                                // sum over species of (nf + 1): triangles, padding
    int *hoff;                                // per species offset into hist
    long long hist_n;
    int *scan_tmp;                            // scratch for the block sums
    const short *chunk_sp;                    // species of each 32-particle chunk
};
void launch_sort(cudaStream_t st, const SortArgs &a);


// Conservation checks (kernels_check.cu).
void launch_charge(cudaStream_t st, bool fp32, long long P, const int *cell, const short *blk_sp, int block,
                   const Species *sp, const Geo64 *geo, const Topo *topo, const void *f0, const void *f1,
                   unsigned long long *q, int N);
void launch_dce(cudaStream_t st, int N, const int *nrp, const int *nedge, const int *ninst,
                const unsigned long long *ifix, const unsigned long long *q0, const unsigned long long *q1, double *out);
// Field probe: E(x_p) = sum_m w_m e[eg_m], w_m = s_m (l_a grad l_b - l_b grad l_a)
// at the probe's barycentrics (a = m+1, b = m+2), precomputed on the host.
struct ProbeW { double w[6]; int eg[3]; int pad; };
void launch_probe(cudaStream_t st, long long n, const ProbeW *pw, const double *e, double2 *ring, long long cap,
                  unsigned long long *count);
void launch_dgl(cudaStream_t st, int N, const int *nrp, const int *nedge, const int *ninst, const double *qunit,
                const double *d, const unsigned long long *q, double *g0, int init, double *out);
long long energy_blocks(int E, int F);
void launch_energy(cudaStream_t st, int E, int F, const long long *hrp, const int *hci, const double *hv,
                   const double *e, const int *einst, const double *b, const Geo64 *geo, const Topo *topo,
                   int ninst, double *part, double *out);

size_t scan_tmp_ints(long long n);
void launch_exclusive_scan(cudaStream_t st, const int *in, int *out, long long n, int *tmp);

// Host-layout particle state into a species range (FP32: barycentrics, u/c).
// cell: the caller's instance-local triangle indices; c2i maps (cell_off +
// caller index) to the internal instance-local index.  Slots [n, cap) of the
// range become padding (triangle -1, load index -1).
void launch_ingest(cudaStream_t st, long long n, long long cap, long long off, int cell_off, int nf, bool fp32,
                   const double *x, const double *u, const int *cell, const int *c2i, const Geo64 *geo,
                   double inv_c, int *cell_o, int *id_o, void *f0, void *f1, void *f2, void *f3, unsigned *status);

// Particle state of a species range [off, off + cap) to load order (FP32
// converts barycentrics to coordinates); i2c maps an internal global triangle
// to the caller's instance-local index.  A slot with triangle -1 and a load
// index in [0, n) is a particle dropped by a write: its entry gets NaN
// position and momentum and triangle -1.
void launch_unsort64(cudaStream_t st, long long n, const int *cell, const int *id, const double *x,
                     const double *y, const double *ux, const double *uy, long long off, long long cap,
                     const int *i2c, double *ox, double *ou, int *oc);
void launch_unsort32(cudaStream_t st, long long n, const int *cell, const int *id, const float *l0,
                     const float *l1, const float *ux, const float *uy, const Geo64 *geo, double c,
                     long long off, long long cap, const int *i2c, double *ox, double *ou, int *oc);

}  // namespace fetdpic

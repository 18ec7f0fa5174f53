/*
 * fetdpic.h - C ABI of the GB300 (sm_103a) charge-conserving relativistic
 * FETD-PIC particle step on 2-D unstructured triangle meshes.
 *
 * Method: Na, Moon, Omelchenko, Teixeira, arXiv:1707.04333.  One time step
 * n -> n+1 of one or many independent instances ("batched" mode) runs, in
 * this order, entirely in CUDA kernels on one GPU:
 *
 *   1. Faraday update   b^{n+1/2} = b^{n-1/2} - dt C e^n            Sec. II.A, Eq. (semi.dis.curl.1)
 *   2. gather           E^n from edge DoFs with Whitney 1-forms,
 *                       B^n = (B^{n+1/2} + B^{n-1/2})/2 from face DoFs
 *                       with Whitney 2-forms                          Sec. II.B, Sec. II.C(a)
 *   3. push             relativistic Boris (with/without tan
 *                       correction), Vay or Higuera-Cary              Sec. II.C, Eqs. (Boris.u1-u4)
 *   4. move + walk      r^{n+1} = r^n + dt u^{n+1/2}/gamma^{n+1/2},
 *                       split into the triangles the segment crosses  Eq. (eq.motion.dis)
 *   5. deposit          i_ab += (Q/dt)(l_a^s l_b^f - l_a^f l_b^s)
 *                       per crossed triangle                          Sec. II.D, Eq. (I.assign)
 *   6. Ampere update    e^{n+1} = e^n + dt M (C^T [*mu^-1] b^{n+1/2} - i^{n+1/2}),
 *                       M = sparse approximate inverse of [*eps]      Sec. II.A, Eq. (semi.dis.curl.2)
 *
 * Conventions (all calls):
 *   - Units are MKS (Sec. I).  2-D TE: E in the plane on edges, B_z on faces,
 *     particle momentum u = gamma v in the plane (m/s).
 *   - Every pointer argument is a HOST pointer unless its comment says
 *     "device".  Inputs are copied during the call; the caller keeps
 *     ownership of every buffer it passes.  Output buffers are allocated by
 *     the caller with the sizes stated.
 *   - Every call returns FETDPIC_OK (0) or a negative fetdpic_status.  On
 *     error, fetdpic_last_error() returns a one-line description.  Device
 *     faults found by the kernels (walk limit, non-finite momentum) are
 *     latched in a device status word and returned by the next
 *     fetdpic_sync / fetdpic_read / fetdpic_check, which clear it: each
 *     latched fault is reported once.
 *   - A context is bound to the CUDA device current at fetdpic_create and to
 *     one CUDA stream; calls on one context are not thread-safe.
 *   - Edges: unless given by the caller, the edges of an instance are all
 *     node pairs (i, j), i < j, of its triangles, oriented i -> j, numbered in
 *     lexicographic order of (i, j).  Triangles are re-ordered
 *     counter-clockwise (nodes 1 and 2 swapped when clockwise); local edge m
 *     is opposite local node m and runs local node m+1 -> m+2 (mod 3).
 *   - Boundary edges (one triangle) are PEC walls: e is held at 0 there and
 *     particles reflect specularly.  The paper does not say how particles
 *     meet a wall; reflection keeps the path continuous, so charge is still
 *     conserved exactly.
 */
#ifndef FETDPIC_H
#define FETDPIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fetdpic_ctx fetdpic_ctx;

typedef enum {
    FETDPIC_OK = 0,
    FETDPIC_EINVAL = -1,     /* bad argument (null pointer, size, index, unknown enum) */
    FETDPIC_ENOMEM = -2,     /* device or host allocation failed */
    FETDPIC_ECUDA = -3,      /* a CUDA runtime call failed (text in fetdpic_last_error) */
    FETDPIC_EMESH = -4,      /* degenerate triangle, non-manifold edge, edge list mismatch */
    FETDPIC_EWALK = -5,      /* a particle crossed more than max_crossings edges in one step */
    FETDPIC_EOUTSIDE = -6,   /* a loaded particle lies in no triangle */
    FETDPIC_ENONFINITE = -7, /* a momentum or position became NaN/Inf */
    FETDPIC_ETIMEOUT = -8,   /* a kernel's bounded wait (staged copies, a grid barrier) gave up:
                                that step is incomplete.  Reporting it discards the current that
                                step deposited and clears the grid-barrier state; particles and
                                fields are those of a partial step, so restore them from a
                                checkpoint (fetdpic_write_particles, fetdpic_write_fields)
                                before stepping on */
    FETDPIC_ESTATE = -9      /* call not valid in the current state */
} fetdpic_status;

typedef enum {
    FETDPIC_BORIS = 0,       /* Sec. II.C(a), t = beta / gamma_bar            */
    FETDPIC_BORIS_TAN = 1,   /* Sec. II.C(a), t = beta_hat tan(|beta|/gamma_bar) */
    FETDPIC_VAY = 2,         /* Sec. II.C(b)                                   */
    FETDPIC_HC = 3           /* Sec. II.C(c), Higuera-Cary                     */
} fetdpic_pusher;

typedef enum {
    /* Plain FP64: global coordinates, same operations in the same order as a
     * plain FP64 evaluation of the paper's formulas (no FMA contraction), so
     * one step from the same state gives bit-identical cells, crossed edges,
     * positions and momenta (Boris-tan excepted: tan is not correctly rounded). */
    FETDPIC_FP64 = 0,
    /* FP32 gather/push/deposit with cell-local barycentric positions and
     * momenta in units of c; FP64 for the Lorentz factor and momentum update
     * of particles with gamma > 10, for the field unknowns e, b, the Faraday
     * update, C^T [*mu^-1] b - i and the checks.  The SPAI product dt M r of
     * the Ampere update runs in FP32 (FP32 matrix values, r rounded to FP32,
     * FP32 sums) and is added to the FP64 e. */
    FETDPIC_FP32 = 1
} fetdpic_precision;

/* Context-wide parameters.  Zero-initialise and set what you need. */
typedef struct {
    double eps0, mu0, c;     /* vacuum constants; 0 = CODATA values */
    int precision;           /* fetdpic_precision */
    int spai_level;          /* sparsity level k >= 1 of the SPAI of [*eps] (Sec. II.A); 0 = 2;
                                -1 = exact inverse (dense, only for <= 4096 free edges) */
    int sort_interval;       /* steps between counting sorts of particles by triangle; 0 = 16, <0 = never */
    int max_crossings;       /* walk limit per particle per step; 0 = 64 */
    int check_interval;      /* every k-th step also computes the continuity and Gauss-law
                                residuals (FP64); 0 = never */
    int record_walk;         /* > 0: keep up to this many crossed edges per particle of the
                                last step (debug / parity; costs bandwidth); 0 = off */
    int block_size;          /* particle-kernel threads per block; 0 = tuned default */
    int use_graphs;          /* 1 = replay steps from a captured CUDA graph; 0 = plain launches */
    int time_stages;         /* 1 = record CUDA events between stages (fetdpic_stage_times) */
    int kernel_variant;      /* FP32 particle kernel, one particle per thread: 2, 3 or 4 =
                                256-thread blocks, that many resident per SM; 5 = particle state
                                staged in shared memory by bulk asynchronous copies; 6 = 128-thread
                                blocks, 7 per SM; 7 = 64-thread blocks, 14 per SM.  Two adjacent
                                particles per thread: 8 = 256-thread blocks, 9 = 128, 10 = 64;
                                11 = 128 and 12 = 64 with the two particles' triangle records read
                                one after the other (fewer registers, 24 warps per SM).  With a
                                per-block deposit window in shared memory (the current of
                                triangles near the block's particles summed there and added to
                                the global current once per block): 13 and 14 = variant 10 with
                                320- and 256-triangle windows, 15 = variant 12 with 192, 16 =
                                variant 9 with 640.  19 = variant 12 compiled for 14 blocks
                                per SM (28 warps); 20 = variant 12 with a 256-triangle window.
                                Hybrids: 17 = variant 12 for the first 6 steps after a sort and
                                variant 14 after them, 18 = the same switching after 4 steps,
                                21 = variant 19 for 6 steps then 14, 22 = variant 19 for 6
                                steps then 20.  0 = default (22).  All give identical results.
                                Other values: FETDPIC_EINVAL. */
    void *cuda_stream;       /* cudaStream_t to run on; NULL = a stream owned by the context */
    /* Optional device allocator (e.g. a framework's caching allocator).  NULL = cudaMalloc/cudaFree. */
    void *(*dev_alloc)(size_t bytes, void *user);
    void (*dev_free)(void *ptr, void *user);
    void *alloc_user;
    long long wait_spin_limit; /* polls of each bounded wait inside a kernel (variant 5's staged
                                copies, the grid barriers of cooperative launches) before it
                                gives up and reports FETDPIC_ETIMEOUT;
                                0 = 2^20; negative = no poll, every such wait gives up at
                                once (exercises the timeout path) */
    int fuse_field_update;   /* 1 = the Ampere update (C^T [*mu^-1] b - i, then the SPAI
                                product) runs as one cooperative launch whose blocks meet at a
                                grid barrier with a bounded wait (FETDPIC_ETIMEOUT if it gives
                                up); 0 = two launches (the default: measured faster on GB300).
                                Same arithmetic, same results. */
} fetdpic_params;

/* One simulation instance (mesh + fields).  Instances share nothing but the
 * kernel launches (block-diagonal packing). */
typedef struct {
    int n_nodes;
    const double *nodes_xy;  /* [n_nodes][2] node coordinates (m) */
    int n_tri;
    const int *triangles;    /* [n_tri][3] node ids in [0, n_nodes) */
    int n_edges;             /* number of rows in `edges`; ignored when edges == NULL */
    const int *edges;        /* optional [n_edges][2] edge list (orientation = e and j sign
                                convention); NULL = derived as described above */
    const int *edge_tags;    /* optional [n_edges] 0 = free, 1 = PEC (e held at 0);
                                NULL = PEC exactly on boundary edges */
    double dt;               /* time step (s) */
    double b0;               /* initial uniform B_z: b_f = b0 * area_f (face DoF, Eq. (B)) */
    double e0x, e0y;         /* initial uniform E on free edges: e_k = E0 . (r_j - r_i) (Eq. (E)) */
    double ext_ex, ext_ey, ext_bz; /* external uniform fields added at each particle */
    /* Optional periodic walls (the paper's Bernstein strip is periodic top and
     * bottom, Sec. III.C): n_periodic node pairs (a, b) in periodic_nodes
     * [n_periodic][2], node b lying at node a + (period_x, period_y) within
     * 1e-9 of the mesh extent.  Each b becomes the same node as its a, so the
     * two copies of a wall edge are one edge (one e unknown, two triangles);
     * a particle crossing it continues from the other copy, translated by the
     * period, with the same momentum.  Requires edges == NULL and
     * edge_tags == NULL (the remaining boundary edges are PEC).  Each node is
     * an image at most once and no triangle may join a node to its image
     * (EMESH).  n_periodic = 0: no periodic walls. */
    int n_periodic;
    const int *periodic_nodes;
    double period_x, period_y;
} fetdpic_instance;

/* Build the mesh topology, incidence matrices C and S~ (Sec. II.A), Whitney
 * geometry, [*eps] (Galerkin edge mass matrix), the diagonal [*mu^-1] =
 * 1/(mu0 A_f), the SPAI M ~ [*eps]^-1 on free edges, and upload everything.
 * inst[n_inst] are host structs; their arrays are copied.  Returns
 * FETDPIC_EMESH for degenerate input.  *out is NULL on error. */
int fetdpic_create(fetdpic_ctx **out, const fetdpic_params *p, int n_inst, const fetdpic_instance *inst);

/* Add one species of n superparticles (charge q, rest mass m) to instance
 * `inst`.  x: [n][2] positions (m); u: [n][2] momenta u = gamma v (m/s),
 * taken as u^{n-1/2} (no half-step back-push): the leapfrog of Eq.
 * (eq.motion.dis) staggers u by half a step against r, and the paper does not
 * say how a loaded state is staggered.  cell_hint: optional [n]
 * triangle indices to try first (a particle goes to the hint when all its
 * barycentric coordinates there are >= 0, else to the lowest-index triangle
 * where they are).  Returns the new species id (>= 0), or FETDPIC_EOUTSIDE if
 * a point lies in no triangle.  Must precede the first fetdpic_step. */
int fetdpic_load_particles(fetdpic_ctx *ctx, int inst, double q, double m, long long n,
                           const double *x, const double *u, const int *cell_hint);

/* Overwrite the state of species `species` (same count as loaded) from host
 * arrays: x [n][2], u [n][2], cell [n] (instance-local triangle of each point,
 * e.g. from a previous fetdpic_read; NULL = locate again on the host).  With
 * `cell` the arrays are copied to the device as they are (fastest from
 * page-locked memory) and converted there, asynchronously on the stream: the
 * host buffers must stay valid until the next fetdpic_sync or read, and a
 * triangle index outside the instance's mesh is found on the device (that
 * particle is dropped: it no longer moves, deposits or counts, the other
 * particles keep their species, and reads return it as missing) and reported
 * as FETDPIC_EINVAL by the next fetdpic_sync or fetdpic_read.  Used for
 * checkpoint/restart and for end-to-end runs that stream the particle state
 * from the host. */
int fetdpic_write_particles(fetdpic_ctx *ctx, int species, const double *x, const double *u, const int *cell);

/* Overwrite the fields of instance `inst`: e [n_edges] (e^n, PEC entries are
 * forced to 0) and b [n_tri] (b^{n-1/2}); either may be NULL. */
int fetdpic_write_fields(fetdpic_ctx *ctx, int inst, const double *e, const double *b);

/* Enqueue nsteps time steps with pusher `pusher` (fetdpic_pusher) on the
 * context stream.  One step is the cycle of Sec. II.A-II.D in the order of
 * the list at the top of this header: Faraday (Eq. (semi.dis.curl.1)),
 * gather (Sec. II.B), push (Sec. II.C), move and walk (Eq.
 * (eq.motion.dis)), deposit (Eq. (I.assign)), Ampere (Eq.
 * (semi.dis.curl.2)); then, every sort_interval steps, the counting sort by
 * triangle (not in the paper).  Asynchronous: returns after the launches;
 * device faults are reported by the next fetdpic_sync. */
int fetdpic_step(fetdpic_ctx *ctx, long long nsteps, int pusher);

/* Wait for the context stream; return the latched device status (walk
 * limit, non-finite momentum, bounded-wait timeout, bad written triangle) of
 * the steps since the last report, then clear it. */
int fetdpic_sync(fetdpic_ctx *ctx);

/* Copy state of instance `inst` to host buffers (each may be NULL), in the
 * staggering of the leapfrog (Sec. II.A, Eq. (eq.motion.dis)): e [n_edges] =
 * e^n, b [n_tri] = b^{n-1/2} (the latest face DoFs), j [n_edges] = i^{n-1/2}
 * of the last step (Eq. (I.assign)).  Then species `species` (ignored
 * if x, u and cell are all NULL): x [n][2], u [n][2], cell [n], in load
 * order.  FP32 mode converts barycentric positions to x = sum_k l_k r_k.  A
 * particle dropped by fetdpic_write_particles reads NaN position and
 * momentum and triangle -1. */
int fetdpic_read(fetdpic_ctx *ctx, int inst, double *e, double *b, double *j,
                 int species, double *x, double *u, int *cell);

/* The particle part of fetdpic_read (x, u, cell of species `species`, load
 * order, same values), without waiting: the state of the species as it is
 * after the work already enqueued on the context stream is copied into a
 * staging area of the species' own (kernel on the context stream), then to
 * the host buffers on a stream of the context's own, while the context stream
 * goes on with later writes, steps or reads.  So the host copy of one step's
 * result can overlap the host-to-device copy of the next step's input.
 *   - No counterpart in the paper: an interface for streaming the state.
 *   - The host buffers (x [n][2], u [n][2], cell [n]; each may be NULL) must
 *     stay valid and untouched until fetdpic_sync returns, which waits for
 *     these copies too; from page-locked memory the copies run at the link's
 *     rate.  Device status words are reported by that sync.
 *   - A second asynchronous read of the same species waits, on the device,
 *     until the first one's host copy has left the staging area.
 *   - The first call allocates the staging areas (36 B per particle of every
 *     species) and the stream.
 * FETDPIC_EINVAL for a bad species; FETDPIC_ENOMEM if the staging cannot be
 * allocated; FETDPIC_ECUDA for a failed launch or copy request. */
int fetdpic_read_particles_async(fetdpic_ctx *ctx, int species, double *x, double *u, int *cell);

/* Same particle output as fetdpic_read (x, u, cell of species `species`, load
 * order, FP32 positions converted), for callers that cannot allocate device
 * memory at the time of the call: real-time loops that forbid allocator
 * latency, plug-ins whose host framework owns all device memory.
 * fetdpic_read allocates its device staging buffer on first use; this call
 * stages through a fixed array compiled into the library instead (9 MiB =
 * 262,144 particles x 36 B; every GPU that loads the library holds it until
 * the process exits) and calls no allocation routine.  Like fetdpic_read it
 * waits for the context stream before it returns.
 *   - The paper has no counterpart: this is an interface convenience.
 *   - Species with more than 262,144 particles are rejected (FETDPIC_EINVAL,
 *     the count in fetdpic_last_error).  The particles must already be on
 *     the device (moving them there allocates): after fetdpic_step,
 *     fetdpic_write_particles, fetdpic_autotune or a fetdpic_read with a
 *     particle buffer; FETDPIC_ESTATE otherwise.
 *   - The first call on each device looks up the array's device address
 *     (with that device current).
 *   - All calls share the one array.  Each call first sets the slots it uses
 *     to all-one bytes, so a particle dropped by fetdpic_write_particles (a
 *     triangle outside the mesh, reported as FETDPIC_EINVAL) reads NaN
 *     position and momentum and triangle -1, never an earlier call's data.
 *     Calls that overlap on the GPU (other threads, other contexts on other
 *     streams) race on the array.
 * x [n][2], u [n][2], cell [n] are host buffers, each may be NULL. */
int fetdpic_read_particles_static(fetdpic_ctx *ctx, int species, double *x, double *u, int *cell);

/* Nodal charge of the current particle state of instance `inst`, Eq.
 * (scatter.charge.assign): q_i = sum_p Q_p lambda_i(r_p) over the particles of
 * the instance, each particle's three barycentric weights rounded to the
 * fixed-point quantum of the instance before the integer sum (the same
 * arithmetic as the continuity and Gauss-law checks).  q [n_nodes] host
 * buffer (C per unit depth; NULL = only the quantum); *quantum (may be NULL)
 * = the charge of one fixed-point unit, so q / quantum are exact integers.
 * With periodic walls the charge of an image node lands on its partner and
 * the image reads 0.  Allocates a device buffer of 8 B per node on the first
 * call; synchronous.  Before the first step it moves the loaded particles to
 * the device like fetdpic_step does. */
int fetdpic_read_charge(fetdpic_ctx *ctx, int inst, double *q, double *quantum);

/* Crossed-edge record of the last step for species `species` (needs
 * record_walk > 0): cnt [n] crossings per particle; rec [n][record_walk]
 * the crossed edges (instance-local ids) in crossing order, a wall
 * reflection stored as -(edge+1).  Load order. */
int fetdpic_read_walk(fetdpic_ctx *ctx, int species, int *cnt, int *rec);

/* Residuals of the latest check step (check_interval > 0), FP64:
 * dce_max = max over nodes of |q^{n+1}-q^n + dt (S~ i^{n+1/2})_k| / (sum of
 * |contributions| at k), the discrete continuity equation (Eq. full.dis.cont);
 * dgl_max = max over nodes of |(S~ d^n - q^n) - (S~ d^0 - q^0)|_k / scale_k,
 * the discrete Gauss law (Eq. semi.dis.div.2) written with the dual flux
 * d^n = d^0 + dt sum (C^T [*mu^-1] b - i) that [*eps] e^n approximates
 * through the SPAI; energy = e.[*eps].e/2 + b.[*mu^-1].b/2 (J per m).
 * Any output may be NULL. */
int fetdpic_check(fetdpic_ctx *ctx, int inst, double *dce_max, double *dgl_max, double *energy);

/* Applied fields that vary in space and time (the synchrocyclotron of
 * Sec. III.A: a magnet over the whole region and an RF field in a gap strip,
 * its frequency following the electrons).  The instance's uniform external
 * fields (ext_ex, ext_ey, ext_bz of fetdpic_instance) act on a particle in
 * triangle f as E = a w_E[f] (ext_ex, ext_ey) and B_z = w_B[f] ext_bz, with
 * a the instance's amplitude (1 until set).
 *
 * fetdpic_set_external_profile: w [n_tri][2] = (w_E, w_B) per triangle of
 * instance `inst` (host array, copied); NULL = all 1.  The first call
 * allocates the weights for all instances (1 elsewhere) and re-captures step
 * graphs.  EINVAL on a non-finite weight.
 *
 * fetdpic_set_external_amplitude: a for the steps enqueued after this call
 * (stream-ordered; steps replayed from graphs see it too).  Returns once the
 * value is on the device.  EINVAL on a non-finite a. */
int fetdpic_set_external_profile(fetdpic_ctx *ctx, int inst, const double *w);
int fetdpic_set_external_amplitude(fetdpic_ctx *ctx, int inst, double amplitude);

/* Initial electrostatic field of a non-neutral load.  The discrete Gauss law
 * (Eq. (semi.dis.div.2)) asks S~ [*eps] e = q of the field; a load whose
 * charges do not cancel needs a starting e that carries them.  With the
 * particles of instance `inst` as loaded by fetdpic_load_particles (before
 * the first step), computes their nodal charge q_i = sum Q lambda_i(r_p)
 * (Eq. (scatter.charge.assign)), solves G^T [*eps] G phi = q on the nodes off
 * the PEC walls (phi = 0 on them; G the node-to-edge incidence, G = -S~^T)
 * by Jacobi-preconditioned conjugate gradients on the host in FP64 (relative
 * residual <= 1e-14), adds e = -G phi to the instance's edge unknowns and
 * restarts the dual flux d = [*eps] e.  From then on the instance's
 * Gauss-law check (fetdpic_check) measures S~ d^n - q^n itself on the nodes
 * off the PEC walls instead of its change since the first step (on wall
 * nodes S~ d - q is the conductor's induced charge and is still compared
 * with its first value); fetdpic_write_fields with an e reverts that.  *iterations and *residual (either may be NULL) report the solve.
 * ESTATE after the first step or on a mesh without PEC walls; EMESH if the
 * solve does not converge. */
int fetdpic_solve_electrostatic(fetdpic_ctx *ctx, int inst, int *iterations, double *residual);

/* Field probes, a diagnostic around the step: the paper reads its relativistic
 * Bernstein-mode spectra off E_x sampled along a line of the domain at every
 * time step, Fourier-transformed in space and time (Sec. III.C).  Registers
 * n points (inst[n] instance of each point, xy [n][2] in metres; host arrays,
 * copied).  After every later step the library evaluates E^{n+1} at each point
 * from the edge unknowns by the Whitney 1-form interpolation of the particle
 * gather (Sec. II.B: E = sum_m s_m e_m (l_a grad l_b - l_b grad l_a)) and
 * stores (E_x, E_y) in a device ring holding the last `capacity` steps; no
 * host transfer per step, and captured step graphs include it.  Replaces any
 * earlier probes and restarts the record; n = 0 removes them.  Errors: EINVAL
 * (bad arguments, n > 2^24 or n * capacity > 1e10), EOUTSIDE (a point in no
 * triangle of its mesh; nothing changes), ENOMEM. */
int fetdpic_set_probes(fetdpic_ctx *ctx, long long n, const int *inst, const double *xy, long long capacity);

/* Waits for the stream and copies the last min(recorded, capacity, max_rows)
 * probe rows, oldest first, into exy [rows][n][2] (caller-owned host buffer).
 * *rows = rows copied, *total = steps recorded since fetdpic_set_probes (either
 * may be NULL).  ESTATE when no probes are set. */
int fetdpic_read_probes(fetdpic_ctx *ctx, double *exy, long long max_rows, long long *rows, long long *total);

/* Sizes of instance `inst`: out[0..5] = n_nodes, n_edges, n_tri, n_free_edges,
 * spai nnz, total particles of the instance. */
int fetdpic_info(fetdpic_ctx *ctx, int inst, long long out[6]);

/* The edge list of instance `inst` as used for e and j: edges [n_edges][2]. */
int fetdpic_read_edges(fetdpic_ctx *ctx, int inst, int *edges);

/* The SPAI of instance `inst` over free edges in CSR with instance-local edge
 * ids: rowptr [n_free+1] (row = free edge in ascending edge id), col [nnz]
 * (edge id), val [nnz]; row_edge [n_free].  Any NULL output is skipped. */
int fetdpic_read_spai(fetdpic_ctx *ctx, int inst, long long *rowptr, int *row_edge, int *col, double *val);

/* Autotuner (no counterpart in the paper, which reports no kernels): times
 * short trials of every (FP32 particle-kernel variant in {2, ..., 12}) x (sort
 * interval in {8, 12, 16, 32}) combination -- only the sort interval for FP64,
 * nothing if sorting is off -- starting each from the current state, keeps
 * the fastest per step (sort cost included), and restores the particle and
 * field state exactly, so the simulation is unchanged: the trials record no
 * probe rows and run no checks, and a device error not yet reported by
 * fetdpic_sync stays pending.  trial_steps <= 0 = 32.  The chosen values are returned in *variant and *sort_interval (each
 * may be NULL) and applied.  Blocks the calling thread. */
int fetdpic_autotune(fetdpic_ctx *ctx, int pusher, int trial_steps, int *variant, int *sort_interval);

/* Change wait_spin_limit of a live context (same meaning as in
 * fetdpic_params); for steps enqueued after the call. */
int fetdpic_set_wait_limit(fetdpic_ctx *ctx, long long wait_spin_limit);

/* Apply a tuning found earlier (e.g. from a cache): variant 0 or 2-12;
 * sort_interval > 0, or < 0 for never. */
int fetdpic_set_tuning(fetdpic_ctx *ctx, int variant, int sort_interval);

/* Device time per stage, summed over every step enqueued since the previous
 * call (needs time_stages = 1; CUDA events recorded on the context stream
 * between stages, read at fetdpic_sync): out[0] Faraday + field record,
 * out[1] particle kernel, out[2] Ampere (C^T H b - i and the SPAI SpMV),
 * out[3] steps timed, out[4] sort, out[5] checks, in ms.  *launches = kernels
 * launched by those steps.  The sums are reset by this call. */
int fetdpic_stage_times(fetdpic_ctx *ctx, double out[6], long long *launches);

/* Algorithmic bytes of one launch of the particle kernel (particle state read
 * and written: FP64 2 x 36 B, FP32 2 x 20 B per particle) and the particle
 * count; the roofline numerator. */
int fetdpic_particle_bytes(fetdpic_ctx *ctx, double *bytes, long long *n_particles);

/* Measurement aid, no counterpart in the paper: the FP32 (fp64 = 0) or FP64
 * (fp64 = 1) fused multiply-add rate of the current device in TFLOP/s, from
 * CUDA-event-timed launches of independent FMA chains filling every SM (best
 * of the launches that ran >= 20 ms; about 0.2 s in all).  It is the
 * denominator of the arithmetic roofline of the FP64 particle path, which the
 * FP64 rate bounds.  Needs no context; runs on a stream of its own. */
int fetdpic_fma_rate(int fp64, double *tflops);

const char *fetdpic_last_error(const fetdpic_ctx *ctx);

void fetdpic_destroy(fetdpic_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FETDPIC_H */

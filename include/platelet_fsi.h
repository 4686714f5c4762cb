/*
 * platelet_fsi.h -- C ABI of the B300 (sm_103a) platelet fluid-structure step.
 *
 * The library computes, per time step, the coupled loop of Wu, Xu, Kim and
 * Alber's multiscale platelet-adhesion model (flow chart of Fig. 1; order
 * stated in Section 3 and at the end of Section 3.4.2):
 *   membrane_forces  hybrid membrane + wall repulsion   (Section 3.1, Eq. 2-11; 3.4.1)
 *   bonds_forces     GPIb-alpha / vWF-A1 bond springs    (Section 3.2, Eq. 14)
 *   ib_spread        Lagrangian force -> lattice force   (Section 3.4.2, Eq. 32, 34-36)
 *   lb_step          D3Q19 BGK + Guo forcing             (Section 3.3, Eq. 16-21)
 *   ib_interp        lattice velocity -> node velocity   (Section 3.4.2, Eq. 31, 33)
 *   bonds_step       Monte-Carlo rupture and formation   (Section 3.2, Eq. 12-13)
 *   sim_step         all of the above, in that order, replayed as CUDA graphs
 *
 * Units: lattice units throughout (spacing h = 1, time step dt = 1, reference
 * density 1).  Grid (nx, ny, nz): x, y periodic; halfway bounce-back walls at
 * z = -1/2 (still) and z = nz - 1/2 (moving with u_top).  Cell (i, j, k) has
 * the linear index (k*ny + j)*nx + i; the cell centre is at (i, j, k).
 *
 * Memory: every device array is owned by the caller (allocate, keep alive,
 * free); the library stores raw pointers in opaque handles and never
 * allocates or frees device memory.  Where a call needs internal storage, a
 * *_query_workspace call gives its size and the caller passes a device block
 * of that size (256-byte aligned).  Host arrays are read during the call only.
 *
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 * Calls only enqueue work, except where stated ("synchronises").
 *
 * Errors: every call returns PFSI_OK (0) or a negative PFSI_ERR_* code;
 * pfsi_last_error() gives a one-line description (per thread).  Argument
 * errors are detected before anything is enqueued.
 */
#ifndef PLATELET_FSI_H
#define PLATELET_FSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PFSI_OK 0
#define PFSI_ERR_ARG (-1)      /* invalid argument (null pointer, bad size, misaligned buffer) */
#define PFSI_ERR_CUDA (-2)     /* a CUDA runtime call or kernel launch failed */
#define PFSI_ERR_CAPACITY (-6) /* a device-side list overflowed (see bonds_status) */
#define PFSI_ERR_UNSTABLE (-7) /* lb_check / sim_check found a non-physical state */
#define PFSI_ERR_TIMEOUT (-8)  /* a bounded device-side wait gave up (see pfsi_wait_selftest) */

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to len).  Returns the length of the full message. */
int pfsi_last_error(char* buf, size_t len);
/* Library version as 10000*major + 100*minor + patch. */
int pfsi_version(void);

/* ===================================================================== *
 * Lattice Boltzmann, Section 3.3
 * ===================================================================== */
#define PFSI_LB_FP32 0  /* populations stored as FP32 f - w_q */
#define PFSI_LB_BF16 1  /* f^neq stored as BF16, (v, rho - 1) as FP32 */
#define PFSI_LB_FP16 2  /* f^neq * 2^fp16_exponent stored as FP16, (v, rho - 1) as FP32 */

typedef struct {
    int nx, ny, nz;   /* grid; each >= 1, nz >= 2 */
    float tau;        /* BGK relaxation time (Eq. 16), > 0.5 */
    float u_top[3];   /* velocity of the top wall; u_top[2] must be 0 */
    float body[3];    /* uniform body-force density added in every cell */
    int storage;      /* PFSI_LB_FP32 (lb_create) or PFSI_LB_BF16 / PFSI_LB_FP16 (lb_create_mixed) */
    int fp16_exponent;/* PFSI_LB_FP16: power-of-two scale of the stored f^neq, -60..60 */
    int walls;        /* PFSI_WALLS_BOUNCEBACK or PFSI_WALLS_ONSITE */
} lb_params;

/* z walls.  BOUNCEBACK: halfway bounce-back, walls at z = -1/2 and
 * nz - 1/2 (moving-wall term at the top).  ONSITE: the velocity walls of
 * Eq. 23-30 (Hecht and Harting) on the node planes k = 0 (still) and
 * k = nz - 1 (moving with u_top): after streaming, the populations entering
 * the fluid there are set so that the node carries the wall velocity (the
 * top wall is the mirror image of the printed bottom case); with a force,
 * the collision velocity is v_w + F/(2 rho) as elsewhere. */
#define PFSI_WALLS_BOUNCEBACK 0
#define PFSI_WALLS_ONSITE 1

typedef struct {
    size_t f_bytes;    /* one population buffer: 19 * n_cells float (FP32) or 16-bit (mixed) */
    size_t g_bytes;    /* force field: n_cells float4 (fx, fy, fz, unused) */
    size_t v_bytes;    /* FP32: velocity field n_cells float4 (vx, vy, vz, rho);
                          mixed: one moments buffer n_cells float4 (vx, vy, vz, rho - 1) */
    size_t flag_bytes; /* row flags: ny * nz uint32 */
    long long n_cells;
} lb_sizes;

typedef struct lb_ctx lb_ctx;

/* Byte sizes of the buffers lb_create needs. */
int lb_query_sizes(const lb_params* p, lb_sizes* out);

/* Creates a lattice on caller-owned device buffers.
 * f_a, f_b: two population buffers, structure of arrays f[q][cell], q in the
 *   paper's D3Q19 numbering (0-based: 0..5 axes +x,-x,+y,-y,+z,-z; 6..17 the
 *   face diagonals in the order fixed by Eq. 23-30; 18 rest).  They hold the
 *   post-collision distribution stored as f - w_q (w_q of Eq. 21).
 * g: force density per cell (float4, w unused).  Must be zero on entry where
 *   the row flag is clear; lb_step zeroes it where it consumed it.
 * v: written by lb_step in flagged rows: (v, rho) with v = u + g/(2 rho).
 * row_flags: one uint32 per (j, k) row; ib_spread sets, ib_interp clears.
 * All buffers 16-byte aligned.  lb_create clears g and the flags (enqueued on
 * the legacy default stream; synchronises). */
int lb_create(const lb_params* p, float* f_a, float* f_b, float* g, float* v,
              uint32_t* row_flags, lb_ctx** out);

/* Mixed-precision storage (p->storage = PFSI_LB_BF16 or PFSI_LB_FP16; no
 * paper counterpart, a storage choice): each cell keeps its (v, rho - 1) in
 * FP32 (m_a/m_b, float4 per cell) and, in 16 bits (fneq_a/fneq_b,
 * [slot][cell]), the deviation of its post-collision populations from
 * E_q = w_q (P + c_q.J + (c_q.J)^2 / 2), J = 3 rho v, P = rho - 1 -
 * 1.5 rho v.v: f*neq_q = f*_q - E_q, which is (1 - 1/tau)(f_q - f_q^eq) +
 * S_q + w_q rho (1 - rho)(3 c_q.v)^2 / 2 (E_q is the equilibrium of Eq. 20
 * but for the last term).  The slots hold the directions grouped by c_z:
 * slots 0..8 = directions 0, 1, 2, 3, 6, 7, 10, 11, 18 (c_z = 0), 9..13 =
 * 4, 8, 12, 14, 16 (c_z = +1), 14..18 = their opposites 5, 13, 9, 17, 15.
 * 108 B per cell per step instead of 152.  A
 * pulling cell rebuilds each incoming population as E_q(source) + f*neq_q.
 * The moments buffer of the current state is the velocity field that
 * ib_interp reads (every cell; no row-flag velocity output).  Same step as
 * lb_create otherwise.  When nx is a multiple of 8 the step moves its tiles
 * with TMA (tensor maps of the four buffers are encoded here; the buffers
 * must stay where they are for the life of the context).  All buffers
 * 16-byte aligned; g and the flags are cleared (synchronises). */
int lb_create_mixed(const lb_params* p, void* fneq_a, void* fneq_b, float* m_a, float* m_b, float* g,
                    uint32_t* row_flags, lb_ctx** out);

/* The current post-collision state as FP32 shifted populations f - w_q,
 * [q][cell], into f_out (device, 19 * n_cells floats): a copy for FP32
 * storage, the reconstruction E_q(rho, v) + f*neq_q for mixed storage. */
int lb_export(lb_ctx* ctx, float* f_out, void* stream);
int lb_destroy(lb_ctx* ctx);

/* Writes the developed shear profile u = u_top (k + 1/2)/nz (bounce-back
 * walls) or u_top k/(nz - 1) (on-site walls), equilibrium plus its
 * first-order non-equilibrium part, post-collision, into the current state.
 * u_top = 0 gives the fluid at rest. */
int lb_init_shear(lb_ctx* ctx, void* stream);

/* nsteps lattice Boltzmann steps (Eq. 16-20): pull streaming with periodic x,
 * y and halfway bounce-back at the z walls (moving-wall term at the top),
 * then BGK collision with Guo's forcing term (Eq. 19, read with the
 * (c c^T - c_s^2 I) tensor and the corrected velocity v).  The force of a
 * cell is body + g where its row is flagged.  Swaps the current buffer. */
int lb_step(lb_ctx* ctx, int nsteps, void* stream);

/* Launch shape of lb_step (no paper counterpart; the result does not depend
 * on it: every shape runs the same per-cell operation sequence and gives
 * bit-identical populations).  FP32 storage: threads per block along x,
 * shape 0..3 = 128, 32, 64, 256 (capped at nx rounded up to 32).  Mixed
 * storage: the kernel and (x, y) column tile of the marching kernels.  nx a
 * multiple of 8: shape 0 = the staged pair kernel (a thread takes two
 * x-adjacent cells, packed FP32x2 arithmetic, each interior plane's 16-bit
 * values copied to shared memory by cp.async) with 64x4 columns, 1 = the
 * pair kernel (global pulls) with 64x4, 2 = the one-cell kernel with 32x8,
 * 3 = the TMA-staged kernel with 32x8 (the one-cell kernel with 32x4 where
 * the driver lacks TMA encoding).  Otherwise: 0, 1 = the pair kernel with
 * 64x4, 64x8; 2, 3 = the one-cell kernel with 32x8, 32x4.  Default 0. */
#define PFSI_LB_SHAPES 4
int lb_set_shape(lb_ctx* ctx, int shape);
int lb_get_shape(const lb_ctx* ctx, int* shape);
/* Autotuner: times every shape over `reps` lattice steps each (CUDA events on
 * `stream`, after one untimed step per shape), keeps the fastest and returns
 * its time per step in *best_ms (may be NULL).  The lattice advances by
 * PFSI_LB_SHAPES * (reps + 1) steps: tune before initialising the state.
 * Synchronises. */
int lb_autotune(lb_ctx* ctx, int reps, void* stream, float* best_ms);

/* Device pointer of the buffer holding the current (post-collision) state
 * (FP32 storage only; mixed storage returns PFSI_ERR_ARG, see lb_export). */
int lb_current(const lb_ctx* ctx, float** f);

/* Device pointer of the velocity field that ib_interp reads, float4 per
 * cell: FP32 storage, the v buffer, (v, rho) valid in the rows flagged at
 * the last step; mixed storage, the current moments buffer, (v, rho - 1) in
 * every cell.  v = u + g/(2 rho) of the last step. */
int lb_velocity(const lb_ctx* ctx, float** v);

/* Sum over all cells of rho and of rho*u (u = momentum of the current
 * post-collision state / rho), accumulated in FP64 on the device into the
 * caller's device scratch dev_scratch4 (4 doubles).
 * out_host[4] = {sum rho, sum rho ux, sum rho uy, sum rho uz}.  Synchronises. */
int lb_moments_fp64(lb_ctx* ctx, double* dev_scratch4, double* out_host, void* stream);

/* Instability check of the current state (no paper counterpart; a
 * diagnostic to call every so many steps): counts the cells whose density or
 * velocity is not finite (or, with 16-bit storage, whose stored f*neq is),
 * whose density is <= 0, and whose speed |u| exceeds u_max (lattice units;
 * the BGK scheme needs |u| well below the lattice speed of sound 1/sqrt(3)).
 * dev_scratch4: caller's device buffer of 4 unsigned 64-bit counters.
 * out_host[3] = {non-finite, rho <= 0, |u| > u_max}.  Returns
 * PFSI_ERR_UNSTABLE if any count is nonzero, PFSI_OK otherwise.
 * Synchronises. */
int lb_check(lb_ctx* ctx, float u_max, unsigned long long* dev_scratch4, long long* out_host, void* stream);

/* ===================================================================== *
 * Immersed boundary, Section 3.4.2 (Eq. 33-36, 4-point cosine kernel)
 * ===================================================================== */
/* g[cell] += F_m phi(x - X_m) phi(y - Y_m) phi(z - Z_m) over the 4x4x4
 * support of every node (Eq. 34-35, h = 1); the support wraps in x, y and is
 * cut at the walls.  Sets the row flags of the cells touched.  A node with a
 * coordinate that is not finite or lies 1e8 lattice units or more from the
 * origin spreads nothing.
 * X: device double[3][M] (structure of arrays), F: device float[3][M]. */
int ib_spread(lb_ctx* ctx, const double* X, const float* F, int M, void* stream);

/* U_m = sum over the support of v phi phi phi (Eq. 33) with v from the last
 * lb_step; if advect != 0, X += U (Eq. 31, forward Euler, dt = 1).  Clears
 * the row flags of the cells visited.  A node with a coordinate that is not
 * finite or lies 1e8 lattice units or more from the origin gets U = NaN and
 * keeps its position.  U: device float[3][M]. */
int ib_interp(lb_ctx* ctx, double* X, float* U, int M, int advect, void* stream);

/* ===================================================================== *
 * Hybrid membrane, Section 3.1 (+ wall repulsion of Section 3.4.1)
 * ===================================================================== */
typedef struct {
    float k_spring;     /* Eq. 2-3 spring constant */
    float k_s, k_t;     /* Eq. 4 global / local area moduli */
    float k_v;          /* Eq. 5 volume modulus */
    float k_b;          /* bending: k_b (1 - cos(theta - theta0)) per edge (Eq. 6 reading) */
    float morse_D;      /* SCE Morse pairs: D[(1 - exp(-a (r - r0)))^2 - 1] */
    float morse_a;
    float rep_F0;       /* wall repulsion F = F0 tau e^{-tau eps}/(1 - e^{-tau eps}) */
    float rep_tau;
    float rep_eps_min;  /* gap clamp */
    float z_wall;       /* wall plane (-1/2) */
} mem_params;

typedef struct mem_ctx mem_ctx;

/* Workspace bytes for a mesh of n_nodes nodes (membrane nodes and interior
 * SCE elements), n_tri outward-oriented triangles tri[3*n_tri] (host), n_pairs
 * Morse pairs and n_plt platelets. */
int membrane_query_workspace(int n_nodes, int n_tri, const int* tri, int n_pairs, int n_plt,
                             size_t* bytes);

/* Builds the per-node gather lists and the rest state (edge lengths, triangle
 * and total areas, volumes, rest dihedral angles, Morse rest distances) from
 * the rest shape X0 (host double[3][n_nodes]) into the device workspace.
 * node_plt: platelet of each node; is_membrane: 1 for surface nodes (wall
 * repulsion), 0 for SCE elements.  pairs: host int[2*n_pairs].  Synchronises. */
int membrane_create(const mem_params* p, int n_nodes, int n_tri, const int* tri, int n_pairs,
                    const int* pairs, int n_plt, const int* node_plt,
                    const unsigned char* is_membrane, const double* X0, void* workspace,
                    size_t ws_bytes, mem_ctx** out);
int membrane_destroy(mem_ctx* ctx);
int membrane_set_params(mem_ctx* ctx, const mem_params* p);

/* F = -grad(H_SCE + H_area + H_volume + H_bend + H_Morse) + F_wall  (Eq. 11,
 * read with the minus sign of Eq. 3).  X: device double[3][n_nodes]; F:
 * device float[3][n_nodes], overwritten.  Two implementations (no paper
 * counterpart; the same per-element arithmetic, summed per node in another
 * order): three passes through per-element force slots in the workspace
 * (the default), or the fused pass, one block per platelet with the
 * platelet's positions and 64-bit fixed-point force accumulators in shared
 * memory (exact sums: forces independent of scheduling), which applies when
 * each platelet's edges, triangles and Morse pairs form one run of the
 * element lists and its nodes fit (about 4,700 nodes). */
int membrane_forces(mem_ctx* ctx, const double* X, float* F, void* stream);
/* path 0 (the default): the three passes; 1: the fused pass where it
 * applies.  membrane_get_path: *fused = 1 if membrane_forces runs the fused
 * pass. */
int membrane_set_path(mem_ctx* ctx, int path);
int membrane_get_path(const mem_ctx* ctx, int* fused);

/* Centroid of every platelet's nodes (membrane and SCE) at positions X:
 * out_dev (device, 4 * n_plt doubles, 8-byte aligned) receives the
 * centroids in its first 3 * n_plt entries ([platelet][x, y, z]); the rest is
 * not written.  FP64 sums in a fixed order (one block per platelet), so
 * repeated calls give identical bits.  Enqueues only. */
int membrane_centroids(mem_ctx* ctx, const double* X, double* out_dev, void* stream);

/* Per-platelet total area and volume of X (FP64 on the device).
 * out_host[2*n_plt] = {S_0, V_0, S_1, V_1, ...}.  Synchronises. */
int membrane_measure(mem_ctx* ctx, const double* X, double* out_host, void* stream);

/* No-allocation variant of membrane_measure.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory (a
 * host application whose own allocator owns every device buffer, or a loop in
 * which cudaMalloc is forbidden) and still want the per-platelet area and
 * volume of a membrane context they have built.  It writes the same
 * out_host[2*n_plt] = {S_0, V_0, ...} as membrane_measure (FP64 sums of the
 * triangle areas and tetrahedron volumes) without using the context's
 * scratch: it accumulates in a library-owned static device array of
 * PFSI_STATIC_MAX_PLATELETS x 2 doubles (128 KiB), which every GPU that loads
 * the library holds until the process exits.  It allocates and frees nothing.
 * Contexts with more than PFSI_STATIC_MAX_PLATELETS platelets are rejected
 * with PFSI_ERR_ARG.  The first call on a device (with that device current)
 * looks up the array's device address and keeps it until the process exits;
 * make that first call before any stream capture, and do not call this entry
 * point after cudaDeviceReset (the reloaded array may live at another address
 * than the one kept).  Every call shares the one array and clears it first: calls that
 * overlap on the GPU (other streams or host threads) race and must be
 * serialised by the caller.  Synchronises on `stream`. */
#define PFSI_STATIC_MAX_PLATELETS 8192
int membrane_measure_static(mem_ctx* ctx, const double* X, double* out_host, void* stream);

/* ===================================================================== *
 * Stochastic adhesion (DAM), Section 3.2
 * ===================================================================== */
typedef struct {
    int lig_i0, lig_j0, lig_ni, lig_nj; /* ligand patch: lattice nodes (i, j) at z = z_wall */
    int box_nx, box_ny;                 /* periodic lengths */
    int max_per_ligand;                 /* receptor sites per vWF (4), 1..32 */
    double z_wall;
    double sigma, l_b, d_capture;       /* Eq. 13-14; 0 < d_capture <= 8 and
                                           2 ceil(d_capture) <= box_nx, box_ny */
    double gamma, kT;                   /* Eq. 12-13 */
    double kon0_dt, koff0_dt;           /* k_on0 dt, k_off0 dt */
    uint64_t seed;                      /* Philox4x32-10 key */
} bond_params;

typedef struct bond_ctx bond_ctx;

int bonds_query_workspace(const bond_params* p, int n_sites, size_t* bytes);

/* Receptor sites are barycentric points: site s lies on triangle
 * site_tri[s] (of tri[3*n_tri]) with weights (w0, w1, 1 - w0 - w1),
 * site_w[2s], site_w[2s+1].  bound[s] = ligand id (j - lig_j0)*lig_ni +
 * (i - lig_i0) or -1; lig_count[l] = bonds of ligand l.  All device arrays. */
int bonds_create(const bond_params* p, int n_sites, const int* site_tri, const double* site_w,
                 const int* tri, int* bound, int* lig_count, void* workspace, size_t ws_bytes,
                 bond_ctx** out);
int bonds_destroy(bond_ctx* ctx);

/* F += bond spring forces (Eq. 14 read as -sigma (|x_b| - l_b) x_b/|x_b|,
 * x_b from the ligand to the receptor), split over the triangle's nodes by
 * the barycentric weights.  X: device double[3][M]; F: device float[3][M]. */
int bonds_forces(bond_ctx* ctx, const double* X, float* F, int M, void* stream);

/* One Monte-Carlo update at time step `step`: rupture of bound sites with
 * P_r = 1 - exp(-k_off dt), Bell k_off (Eq. 12); then each site free at the
 * start of the step tests every ligand within d_capture (minimum image in
 * x, y) and below capacity with P_f = 1 - exp(-k_on dt), k_on of Eq. 13,
 * proposing to the lowest ligand id that succeeded; each ligand accepts
 * proposals in ascending site id up to max_per_ligand.  Uniforms come from
 * Philox4x32-10 keyed by seed with counter (site, step lo, step hi,
 * purpose): purpose 0 rupture; a candidate ligand at node (i0 + di,
 * j0 + dj), (i0, j0) = floor of the site's wrapped (x, y), r =
 * ceil(d_capture), di and dj in 1 - r .. r, draws with purpose
 * 1 + (dj + r - 1) 2r + (di + r - 1) (for d_capture <= 1: 1 + 2 dj + di). */
int bonds_step(bond_ctx* ctx, const double* X, int M, uint64_t step, void* stream);

/* Cumulative event counts and overflow status.  out_host[3] = {ruptures,
 * formations, overflowed proposals}.  Synchronises.  A nonzero overflow means
 * a ligand received more than 64 proposals in one step (then only the first
 * 64 in arrival order were considered) and returns PFSI_ERR_CAPACITY. */
int bonds_status(bond_ctx* ctx, long long* out_host);

/* --------------------------------------------------------------------- *
 * Tether (pause-time) tracking (Section 4.2).  Reading: a platelet is
 * tethered after a step's adhesion update when at least one of its
 * receptor sites holds a wall bond; a tether event runs from the first such
 * update to the first later update after which it holds none, and its pause
 * time is the number of updates it spanned (a bond that forms in step s and
 * breaks in step s + 2 gives a pause of 2 steps).  One block per platelet
 * counts its bound sites in a fixed order and updates, on the device:
 *   state[p]   the step count at which platelet p's current tether began,
 *              or -1 when it is free (caller-owned int64 [n_plt]; initialise
 *              it to -1, or to a saved state when a run continues);
 *   pauses[]   completed pause times in steps, appended in no fixed order
 *              (caller-owned int64 [capacity]);
 *   count[0]   the number of completed events (caller-owned uint64; events
 *              past `capacity` are counted but not stored).
 * "Step count" is the number of completed steps: after the update of step s
 * it is s + 1. */
typedef struct tether_ctx tether_ctx;

/* Workspace bytes for n_sites sites on n_plt platelets. */
int tether_query_workspace(int n_sites, int n_plt, size_t* bytes);

/* site_plt: host int32 [n_sites], the platelet of every site of `bonds`
 * (0 <= site_plt < n_plt).  ws: device workspace of tether_query_workspace
 * bytes (the per-platelet site lists).  The context keeps the pointers of
 * bonds, state, pauses and count (all caller-owned).  Synchronises. */
int tether_create(const bond_ctx* bonds, int n_plt, const int* site_plt, void* ws, size_t ws_bytes, long long* state,
                  long long* pauses, int capacity, unsigned long long* count, tether_ctx** out);
int tether_destroy(tether_ctx* ctx);

/* Update after the bonds_step of step `step` (the step count is step + 1).
 * In a simulation (sim_set_tether) the update runs inside the step after the
 * adhesion update instead. */
int tether_update(tether_ctx* ctx, uint64_t step, void* stream);

/* ===================================================================== *
 * Platelet-platelet bridges GPIb-alpha - vWF - GPIb-alpha (Section 3.2)
 *
 * The paper models these bonds like the wall bonds and prints no equations
 * for them.  Reading: a plasma vWF joins two receptor sites on different
 * platelets; the bridge is one linear spring between the two sites (the
 * form of Eq. 14) with its own spring constant, rest length and capture
 * distance, and the rates of Eq. 12 (rupture) and Eq. 13 (formation).  A
 * site holds at most one bond of either kind.  Per step, after the wall
 * update (bonds_step):
 *   rupture    every bridge i < j breaks with P_r = 1 - exp(-k_off dt),
 *              k_off = k_off0 exp(gamma F_b / kT), F_b = sigma |x_b - l_b|;
 *              its sites stay free until the next step;
 *   formation  every pair i < j of free sites (no wall bond, no bridge) on
 *              different platelets with |x_i - x_j| < d_capture succeeds
 *              with P_f = 1 - exp(-k_on dt), k_on of Eq. 13; each site picks
 *              its lowest-index successful partner; a bridge forms where two
 *              sites picked each other.
 * Draws: Philox4x32-10 with counter (i, j, step lo, purpose) and key
 * (seed lo, seed hi ^ step hi), i < j; purpose 16 rupture, 17 formation.
 * Pair vector x_i - x_j (i < j), minimum image in x, y, FP64.  The outcome
 * does not depend on thread scheduling.
 * ===================================================================== */
typedef struct {
    double sigma, l_b, d_capture;       /* bridge spring, rest length, capture distance */
    double gamma, kT;                   /* Eq. 12-13 */
    double kon0_dt, koff0_dt;           /* k_on0 dt, k_off0 dt */
    int box_nx, box_ny;                 /* periodic lengths */
    uint64_t seed;                      /* Philox4x32-10 key */
} bridge_params;

typedef struct bridge_ctx bridge_ctx;

/* Workspace bytes for n_sites receptor sites, n_plt platelets and M nodes. */
int bridges_query_workspace(const bridge_params* p, int n_sites, int n_plt, int M, size_t* bytes);
/* Bridges between the receptor sites of `bonds` (its site_tri, site_w, tri
 * and bound arrays).  node_plt: host int[M], the platelet of each node; the
 * nodes of each platelet must be contiguous (PFSI_ERR_ARG otherwise).
 * partner: caller-owned device int[n_sites], the other site of each bridge
 * or -1 (symmetric; -1 everywhere to start).  The wall bonds of `bonds`
 * skip bridged sites from now on; destroy the bridges before the bonds.
 * ws: bridges_query_workspace bytes, 256-byte aligned.  Synchronises. */
int bridges_create(const bridge_params* p, bond_ctx* bonds, int n_plt, const int* node_plt, int M, int* partner,
                   void* workspace, size_t ws_bytes, bridge_ctx** out);
int bridges_destroy(bridge_ctx* ctx);
/* F += bridge spring forces: on site i, -sigma (|d| - l_b) d/|d| with
 * d = x_i - x_partner, the opposite on the partner, split over each site's
 * triangle nodes by the barycentric weights.  X: device double[3][M];
 * F: device float[3][M]. */
int bridges_forces(bridge_ctx* ctx, const double* X, float* F, int M, void* stream);
/* One Monte-Carlo update of the bridges at time step `step` (after the wall
 * update of the same step).  Enqueues 6 kernels and a memset. */
int bridges_step(bridge_ctx* ctx, const double* X, int M, uint64_t step, void* stream);
/* Cumulative counts, out_host[3] = {ruptures, formations, neighbour-list
 * overflows (a platelet near more than 16 others: all its free sites were
 * tested, so only the pruning was lost)}.  Synchronises. */
int bridges_status(bridge_ctx* ctx, long long* out_host);
/* The partner array given at create. */
int bridges_partner(bridge_ctx* ctx, int** partner_dev);

/* ===================================================================== *
 * Finite-element bending, Section 3.1 (Eq. 6-10)
 *
 * The membrane is covered by quadratic six-node triangles (Eq. 7):
 * elem6[6 e + 0..2] are an element's corners, counter-clockwise seen from
 * outside (parametric (0,0), (1,0), (0,1)), elem6[6 e + 3..5] the nodes at
 * the midpoints of edges 0-1, 1-2, 2-0.  One evaluation:
 *   1. unit normal at every element node, averaged over the elements sharing
 *      the node (sum of unit normals, normalised);
 *   2. Eq. 9 at every element node: [dX/dxi; dX/deta; n] kappa =
 *      [dn/dxi; dn/deta; 0] with the nodal normals interpolated by Eq. 7;
 *      K = tr(kappa)/2 (Eq. 10) and K_G = kappa_1 kappa_2, each averaged
 *      (plain mean) over the elements sharing the node;
 *   3. Lap_S K: the surface gradient of K by the same system, averaged per
 *      node, then its surface divergence, averaged per node;
 *   4. F_i = A_i (k0/2) (Lap_S K + 2 K (K^2 - K_G)) n_i: the first variation
 *      of H = (k0/2) int K^2 dS (Eq. 6).  The force printed after Eq. 10
 *      lacks k0/2 and the Gaussian-curvature term, without which a sphere
 *      would not be force-free.  A_i: one third of each of the flat
 *      sub-triangles (0,3,5), (3,1,4), (5,4,2), (3,4,5) that touch node i.
 * FP32 arithmetic in coordinates relative to each element's first corner;
 * the node averages are fixed-order sums (deterministic).  Nodes of no
 * element (SCE elements) get no force.
 * ===================================================================== */
typedef struct fem_ctx fem_ctx;

/* Workspace bytes for n_nodes nodes and n_elem six-node elements. */
int fem_query_workspace(int n_nodes, int n_elem, size_t* bytes);
/* Builds the node -> element-node lists on the host and copies them and
 * elem6 (host int[6*n_elem]) into the device workspace (caller-owned,
 * 256-byte aligned, fem_query_workspace bytes; kept until fem_destroy).
 * Rejects node indices outside [0, n_nodes) and elements with a repeated
 * node (PFSI_ERR_ARG).  Synchronises. */
int fem_create(int n_nodes, int n_elem, const int* elem6, void* ws, size_t ws_bytes, fem_ctx** out);
int fem_destroy(fem_ctx* ctx);
/* X: device double[3][n_nodes]; F: device float[3][n_nodes], overwritten
 * (accumulate = 0) or added to.  Enqueues 8 kernels on `stream`. */
int fem_bending_forces(fem_ctx* ctx, float k0, const double* X, float* F, int accumulate, void* stream);
/* Diagnostics of the same passes: fields (device float[7][n_nodes])
 * receives n_x, n_y, n_z, A, K, K_G, Lap_S K per node. */
int fem_fields(fem_ctx* ctx, const double* X, float* fields, void* stream);

/* ===================================================================== *
 * Learned membrane surrogate (no paper counterpart)
 *
 * A per-node network 42 -> 128 -> 128 -> 18 (GELU, tanh form) sets the
 * element stresses of the local membrane terms of Section 3.1: edge springs
 * (Eq. 2-3), the local area term (Eq. 4, second term) and dihedral bending.
 * The global area term, volume (Eq. 5), Morse pairs and wall repulsion stay
 * exact.  The local energy is split into node shares: node i with one-ring
 * n_0..n_{d-1} (3 <= d <= 6, counter-clockwise seen from outside, starting at
 * the neighbour of smallest index) owns, per slot k, half the spring of the
 * spoke (i, n_k), a third of the area term of the fan triangle
 * (i, n_k, n_{k+1}) and half the bending of the spoke (torsion of the chain
 * n_{k+1} - i - n_k - n_{k-1}).  Its 18 element strains are
 * x_s = (L - L0)/L0, x_a = (S - S0)/S0 and x_b = phi - phi0; the network sees
 * their direction x * in_scale / |x * in_scale| (inputs 0..17: six
 * stretches, six area strains, six bending angles) and the rest descriptors
 * L0/l, S0/l^2, cos phi0, sin phi0 of each slot ((r - in_shift) * in_scale,
 * inputs 18..41; l = mean rest spoke length), zero for empty slots.  Its
 * output o sets the stresses y = x * m * out_scale * o with the rest moduli
 * scales m = (L0^2, S0, 1), and the local force is
 * F = - sum_i sum_j y_j dx_j/dX (exact strain gradients; each row adds to its
 * node and its one-ring with atomic adds).  The exact stresses are
 * (k_spring/2) L0^2 x_s, (k_t/3) S0 x_a and (k_b/2) sin x_b.
 *
 * Parameters: one caller-owned device buffer of PFSI_SG_PARAM_BYTES
 * (256-byte aligned): PFSI_SG_N_FLOATS floats at offset 0 (the trained block
 * of PFSI_SG_N_TRAINED floats, then in_shift[64], in_scale[64],
 * out_scale[32], tgt_scale[32]), then at the next 256-byte boundary the BF16
 * copies the tensor cores read (refresh with sg_sync_shadows after writing
 * the floats).  Weights are row-major [outputs][inputs]; padding rows and
 * columns (inputs 42..63, outputs 18..31) must be zero and stay zero under
 * training.
 * ===================================================================== */
#define PFSI_SG_IN 42
#define PFSI_SG_IN_PAD 64
#define PFSI_SG_HID 128
#define PFSI_SG_OUT 18
#define PFSI_SG_OUT_PAD 32
#define PFSI_SG_W1 0          /* [128][64] */
#define PFSI_SG_B1 8192       /* [128] */
#define PFSI_SG_W2 8320       /* [128][128] */
#define PFSI_SG_B2 24704      /* [128] */
#define PFSI_SG_W3 24832      /* [32][128] */
#define PFSI_SG_B3 28928      /* [32] */
#define PFSI_SG_N_TRAINED 28960
#define PFSI_SG_IN_SHIFT 28960  /* [64] */
#define PFSI_SG_IN_SCALE 29024  /* [64] */
#define PFSI_SG_OUT_SCALE 29088 /* [32] */
#define PFSI_SG_TGT_SCALE 29120 /* [32] */
#define PFSI_SG_N_FLOATS 29152
#define PFSI_SG_PARAM_BYTES 215040
#define PFSI_SG_BF16 0  /* BF16 operands on the tensor cores (tcgen05), FP32 accumulation */
#define PFSI_SG_FP32 1  /* FP32 on CUDA cores: check mode */

typedef struct sg_ctx sg_ctx;

int sg_params_bytes(size_t* bytes);
/* Rewrites the BF16 copies of W1, W2, W3 (and the transposed copies the
 * backward pass reads) from the FP32 block. */
int sg_sync_shadows(void* params, void* stream);

/* Training.  feat: [batch][64] inputs (BF16 for PFSI_SG_BF16, float for
 * PFSI_SG_FP32; 16-byte aligned), target: float [batch][36], per row
 * a[18] then b[18] (sg_targets), batch a multiple of 128 (pad with zero
 * rows: they add nothing to the gradients but count in the mean).  Writes
 * grad (PFSI_SG_N_TRAINED floats, the trained-block layout) and, if loss is
 * not NULL, the device double *loss = mean over the batch and the 18
 * outputs of (a o - b)^2.  work: sg_query_work(batch) bytes, 256-byte
 * aligned.  Deterministic (fixed reduction order). */
int sg_query_work(int batch, size_t* bytes);
int sg_grad(const void* params, const void* feat, const float* target, int batch, int mode, float* grad,
            double* loss, void* work, size_t work_bytes, void* stream);
/* Device error flag of the last sg_grad on this workspace (1: a bounded wait
 * on the tensor cores gave up).  Synchronises. */
int sg_work_status(void* work, int batch, int* flag);
/* One Adam step (Kingma and Ba) of the trained block with moments m, v
 * (PFSI_SG_N_TRAINED floats each, zero before the first step), step count
 * t >= 1; refreshes the BF16 copies. */
int sg_adam(void* params, const float* grad, float* m, float* v, float lr, float beta1, float beta2, float eps,
            int t, void* stream);

/* Mesh context: one-rings and rest one-ring data of the membrane nodes
 * (nodes of the triangles; is_membrane may be NULL), computed on the host in
 * FP64 from X0 (double[3][n_nodes]); tri int[3*n_tri] outward oriented, each
 * one-ring closed with 3..6 neighbours.  mode: PFSI_SG_BF16 or PFSI_SG_FP32
 * for sg_membrane_forces.  ws: sg_query_workspace(n_nodes) bytes, 256-byte
 * aligned, caller-owned (also holds the inference activations). */
int sg_query_workspace(int n_nodes, size_t* bytes);
int sg_create(int n_nodes, int n_tri, const int* tri, const double* X0, const unsigned char* is_membrane, int mode,
              void* ws, size_t ws_bytes, sg_ctx** out);
int sg_destroy(sg_ctx* ctx);
/* Number of surrogate nodes (rows) and, optionally, the device array of their
 * node ids (rows padded to a multiple of 128 with -1). */
int sg_rows(const sg_ctx* ctx, int* rows, const int** node);
/* Inputs of every surrogate node at positions X (double[3][n]) into feat
 * ([rows][64]; BF16 or float by the context's mode; NULL: the context's own
 * buffer), its element strains into xs (float [rows][18]; NULL: own) and the
 * rest moduli scales (L0^2, S0, 1) into ms (float [rows][18]; NULL: own). */
int sg_features(sg_ctx* ctx, const void* params, const double* X, void* feat, float* xs, float* ms, void* stream);
/* F = exact global terms + surrogate local forces: Morse pairs (and, on a
 * mesh with Morse pairs, the wall term) by the plain passes, the global area
 * and volume forces (Eq. 4-5, the platelet coefficients from the plain
 * triangle sums) per node from its fan in the surrogate kernel, which also
 * adds the wall term on a mesh without Morse pairs.  F is overwritten. */
int sg_membrane_forces(sg_ctx* ctx, const void* params, mem_ctx* mem, const double* X, float* F, void* stream);
/* Training record of every row from its strains xs and moduli scales ms
 * (sg_features; NULL: the context's own) and the membrane coefficients of
 * the local terms: the exact stresses y (k_spring/2 L0^2 x_s, k_t/3 S0 x_a,
 * k_b/2 sin x_b) give target[r] = (a[18], b[18]) with a = x m tgt_scale and
 * b = y tgt_scale / out_scale; float [rows][36]. */
int sg_targets(const sg_ctx* ctx, const void* params, float k_spring, float k_t, float k_b, const float* xs,
               const float* ms, float* target, void* stream);
/* Device error flag of the context's tensor-core kernels.  Synchronises. */
int sg_status(const sg_ctx* ctx, int* flag);

/* Diagnostic of the bounded device waits (no paper counterpart): one thread
 * waits, with at most `limit` polls, for an mbarrier phase that nothing
 * completes, using the same bounded wait the tensor-core kernels use for
 * their MMA completion (whose timeouts they report through sg_status /
 * sg_work_status).  Nothing asynchronous is in flight, so giving up is safe.
 * dev_word: caller's device int.  Returns PFSI_ERR_TIMEOUT when the wait gave
 * up (the expected outcome), PFSI_OK if the phase completed.  Synchronises. */
int pfsi_wait_selftest(int limit, int* dev_word, void* stream);

/* ===================================================================== *
 * Coupled step (Fig. 1)
 * ===================================================================== */
typedef struct sim_ctx sim_ctx;

/* Ties a lattice, a membrane mesh and a bond set to the node arrays
 * X (double[3][M]), F, U (float[3][M]).  bonds may be NULL (no adhesion).
 * first_step is the step index of the first sim_step (Philox counter).
 * With bonds, allocates and fills (synchronously) the platelet of each
 * receptor site and of each block of 256 sites, and a per-platelet flag that
 * each step's adhesion update sets for the platelets whose every node lies
 * beyond the capture distance above the wall: their sites make no proposal
 * (the per-site test would reject each of them, so the bond events are
 * unchanged; Section 3.2). */
int sim_create(lb_ctx* lb, mem_ctx* mem, bond_ctx* bonds, double* X, float* F, float* U, int M,
               uint64_t first_step, sim_ctx** out);
int sim_destroy(sim_ctx* ctx);

/* nsteps coupled steps: membrane_forces, bonds_forces, ib_spread, lb_step,
 * ib_interp with advection, bonds_step.  The sequence of one step is captured
 * once into a CUDA graph per lattice-buffer parity and replayed. */
int sim_step(sim_ctx* ctx, int nsteps, void* stream);

/* nsteps coupled steps, recording the node positions of every step: after
 * step k, X (double[3][M]) is copied into slot k % ring of dev_ring (device,
 * ring * 3M doubles) on `stream`, then from there into slot k % ring of
 * host_ring (pinned host memory, ring * 3M doubles) on a copy stream of the
 * context, so the device-to-host copy overlaps the next step; a slot is
 * reused only after its previous copy finished.  2 <= ring <= 64.  Returns
 * after enqueueing; `stream` is ordered after the last copy (synchronise it
 * before reading host_ring; slot k % ring then holds step k of the last
 * `ring` steps). */
int sim_step_record(sim_ctx* ctx, int nsteps, double* dev_ring, double* host_ring, int ring, void* stream);

/* nsteps coupled steps, following the platelets: after step k the
 * centroids of all platelets (the mean node position of each, computed
 * inside the step graphs from FP64 sums that the interpolation pass forms
 * per chunk of nodes, added in a fixed order) are copied to
 * host_out[k][n_plt][3] (pinned host memory,
 * nsteps * 3 * n_plt doubles) on the context's copy stream, overlapping the
 * next steps.  Steps run eight per graph where they can (one strided copy per
 * eight steps), one per graph otherwise.  dev_scratch: device, 72 * n_plt
 * doubles (18 slots of 4 * n_plt), kept by the context's graphs until another
 * scratch is passed.  Returns after enqueueing; `stream` is ordered after the
 * last copy. */
int sim_step_track(sim_ctx* ctx, int nsteps, double* dev_scratch, double* host_out, void* stream);

/* Index of the next step (first_step + steps taken). */
int sim_step_index(const sim_ctx* ctx, uint64_t* out);

/* Uses the surrogate for the membrane forces of every following step
 * (sg_membrane_forces in place of membrane_forces); sg = NULL returns to
 * the plain solver (the fallback).  The graphs are recaptured. */
int sim_set_surrogate(sim_ctx* ctx, sg_ctx* sg, const void* params);

/* Adds the finite-element bending force (fem_bending_forces with modulus k0)
 * to the membrane forces of every following step; give the membrane context
 * k_b = 0 so that the dihedral term is not counted twice.  fem = NULL removes
 * it.  The mesh must have the simulation's node count.  The graphs are
 * recaptured. */
int sim_set_fem_bending(sim_ctx* ctx, fem_ctx* fem, float k0);

/* lb_check of the simulation's lattice plus a scan of the node positions:
 * out_host[4] = {non-finite cells, rho <= 0, |u| > u_max, node coordinates
 * (entries of X) that are not finite or lie 1e8 lattice units or more from
 * the origin}.  Nodes with such a coordinate take no part in spreading and
 * interpolation (their support cells would overflow the cell indices): ib_interp
 * sets their velocity to NaN and leaves their position as it is.  Returns
 * PFSI_ERR_UNSTABLE if any count is nonzero.  dev_scratch4 as for lb_check.
 * Synchronises. */
int sim_check(sim_ctx* ctx, float u_max, unsigned long long* dev_scratch4, long long* out_host, void* stream);

/* Adds the platelet-platelet bridges to every following step: their spring
 * forces after the wall bond forces, their update after the wall update.
 * The bridges must be built on the simulation's bond context; their step
 * counter continues from the simulation's.  br = NULL removes them.  The
 * graphs are recaptured.  Synchronises. */
int sim_set_bridges(sim_ctx* ctx, bridge_ctx* br);

/* Track tethers (pause times) in the step: the update of `tr` (whose bonds
 * must be the simulation's) runs after every step's adhesion update; null
 * turns tracking off.  The step graphs are rebuilt on the next step. */
int sim_set_tether(sim_ctx* ctx, tether_ctx* tr);

/* Measurement aid (no paper counterpart): on != 0 records two CUDA events
 * around the lattice Boltzmann kernel inside the step graph (the graphs are
 * recaptured), so that each step measures that kernel where it runs, inside
 * the coupled step.  on = 0 removes them. */
int sim_time_lb(sim_ctx* ctx, int on);
/* Milliseconds between those two events in the most recent step.
 * Synchronises on the second event. */
int sim_lb_ms(sim_ctx* ctx, float* ms);

/* ===================================================================== *
 * Batches of independent chambers (no paper counterpart)
 * ===================================================================== */
typedef struct lb_batch lb_batch;

/* A batch of n lattices of any sizes and storage modes (all at the same
 * buffer parity; the lattices stay owned by the caller and must outlive the
 * batch).  lb_batch_step advances every lattice by one lb_step per step with
 * ONE kernel launch per storage mode present: the cells of all lattices are
 * cut into tiles (FP32: 256 consecutive cells in x-fastest order, 256-thread
 * blocks; mixed storage: (x, y) columns over up to 16 planes, 128-thread
 * blocks, the column shape picked per lattice), listed lattice after
 * lattice, and a persistent grid of as many blocks as are resident on the
 * GPU at once walks the list.  Every tile runs the per-cell arithmetic of
 * lb_step, so each lattice's populations are bit-identical to lb_step on it
 * alone.  The initial column shape of a mixed lattice is the one with the
 * fewest threads counting idle ones in ragged columns (and a quarter per
 * ring cell). */
int lb_batch_create(lb_ctx* const* lattices, int n, lb_batch** out);
int lb_batch_destroy(lb_batch* b);
int lb_batch_step(lb_batch* b, int nsteps, void* stream);
/* Autotuner of the batch: for each mixed-storage lattice, times every
 * column shape on that lattice alone (`reps` launches after one untimed
 * launch, CUDA events on `stream`) and keeps the fastest; then, per storage
 * mode, times the batched launch with 1 .. (resident blocks) blocks per SM
 * and keeps the fastest grid (until lb_batch_set_grid); returns in
 * *ms_per_step (may be NULL) the time of one batched step.  The timed
 * launches read the current buffers and write the others without advancing
 * the parity, so the state is left unchanged as long as no spread force is
 * pending (g zero: true after lb_init_shear and between coupled steps; the
 * step that consumes g clears it).  Synchronises. */
int lb_batch_autotune(lb_batch* b, int reps, void* stream, float* ms_per_step);
/* Grid of the batched launches: blocks_per_sm blocks per SM (0, the
 * default: every block that fits, so the grid is persistent over the tile
 * list; fewer leave SM slots to kernels on other streams).  No effect on
 * results. */
int lb_batch_set_grid(lb_batch* b, int blocks_per_sm);
/* Column shape per lattice (0: the pair kernel's 64x4, 1: the one-cell
 * kernel's 32x4, 2: its 16x8; -1 for FP32):
 * shapes[n] read or set (set ignores the FP32 entries; an entry outside
 * 0..2 for a mixed lattice is PFSI_ERR_ARG and changes nothing).  The
 * shapes do not change any cell's arithmetic. */
int lb_batch_get_shapes(const lb_batch* b, int* shapes);
int lb_batch_set_shapes(lb_batch* b, const int* shapes);

typedef struct batch_ctx batch_ctx;

/* A batch of n chambers, each a sim_ctx of its own (own lattice, mesh,
 * bonds, parameters; all at the same lattice-buffer parity).  batch_step
 * replays one CUDA graph that holds steps_per_graph steps of every chamber.
 * The chambers are dealt into groups of about equal cell counts (largest
 * lattice first, each to the group with the fewest cells so far; one group
 * unless batch_set_layout says otherwise), each group an independent chain
 * of the graph.  Per step of a group whose chambers have no learned
 * surrogate, finite-element bending, bridges or tethers, EVERY kernel of the
 * step is one launch for all the group's chambers: membrane passes, bond
 * forces, spreading, the lattice step (one batched launch per storage mode,
 * as lb_batch_step), interpolation, bond rupture, proposal and resolution.
 * A group with such a chamber runs each chamber's kernels before and after
 * the lattice step on parallel branches (greatest stream priority; the
 * lattice launches take the least, so the branches' kernels get freed SM
 * slots first).  Each
 * chamber's results are those of sim_step on it alone (spreading sums up to
 * the order of its FP32 atomics).  The sims stay owned by the caller and
 * must outlive the batch; stepping one on its own makes the next batch_step
 * fail (PFSI_ERR_ARG: the lattice-buffer parities differ). */
int batch_create(sim_ctx** sims, int n, int steps_per_graph, batch_ctx** out);
int batch_destroy(batch_ctx* ctx);
/* nsteps (a multiple of steps_per_graph) steps of every chamber. */
int batch_step(batch_ctx* ctx, int nsteps, void* stream);
/* Layout of the step graph (no effect on results): `groups` chamber groups
 * (>= 1, capped at n) and the lattice launches' grid, blocks_per_sm blocks
 * per SM (0: every block that fits, a persistent grid over the tile list).
 * Resets the column shapes to their defaults (batch_autotune picks them);
 * the graphs are captured again at the next batch_step. */
int batch_set_layout(batch_ctx* ctx, int groups, int blocks_per_sm);
/* lb_batch_autotune on each group's lattices (between steps: the state is
 * unchanged); *lb_ms_per_step = the sum of the groups' batched lattice step
 * times.  The graphs are captured again at the next batch_step.
 * Synchronises. */
int batch_autotune(batch_ctx* ctx, int reps, void* stream, float* lb_ms_per_step);

#ifdef __cplusplus
}
#endif
#endif

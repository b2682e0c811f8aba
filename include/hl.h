/*
 * hl.h -- C ABI of the GB300 Hermite-leapfrog solver (libhl.so).
 *
 * Method: Vargas, Hagstrom, Chan, Warburton, "Leapfrog time-stepping for
 * Hermite methods", arXiv 1808.10481.
 *
 * The solver advances the first-order acoustics system
 *     p_t + div u = 0,   u_t + grad p = 0            (unit wave speed)
 * on the periodic unit box [0,1)^dim.  This is the paper's system
 * p_t = c div v, v_t = c grad p (Section 2, eq. waveModel; Section 3.1.2,
 * eq. wavend) with c = 1 and v = -u, and the sign form of its experiments
 * (Section 4, Section 5, Section 6).
 *
 * Grids and data (Section 2, eqs. pGrid and dGrid; Section 5):
 *   - each axis k has n_k nodes per grid and spacing h_k = 1/n_k;
 *   - primal node j sits at j*h_k and carries p; dual node j sits at
 *     (j + 1/2)*h_k and carries all dim velocity components;
 *   - every node carries the scaled derivatives
 *         f~_a = prod_k h_k^{a_k} / a_k! * d^a f,   0 <= a_k <= m,
 *     i.e. nq = (m+1)^dim values per node per field component;
 *   - p is held at t = n*dt and u at t = (n + 1/2)*dt (Section 2: the
 *     staggered start, p at t0 and v at t0 + dt/2).
 *
 * One step (Section 2, eqs. update1, LFloop, final1; Section 3.1.2, eqs. pdup
 * and vdup; Section 5, eq. lf1update2D): for every primal node, build the
 * tensor-product Hermite-Birkhoff interpolant of degree 2m+1 per axis of u
 * on the cell whose 2^dim vertices are the surrounding dual nodes (Section 2,
 * eq. interp), evaluate its exact Cauchy-Kowalevsky evolution at the node over
 * +-dt/2 and update p (the p-half); then do the same for every dual node with
 * the interpolant of the new p and update u (the u-half).
 *
 * HOST LAYOUT (hl_set_initial, hl_get_fields):
 *   p[node][q], u[comp][node][q], row-major double, with
 *   node = ix + n_0*(iy + n_1*iz) and q = a_0 + (m+1)*(a_1 + (m+1)*a_2).
 * DEVICE LAYOUT (hl_bind_device, hl_set_initial_device, hl_get_fields_device
 * use the host layout; hl_bind_device uses this one):
 *   p[q][node], u[comp][q][node] ("slot-major"), double.
 *
 * Errors: every int-returning call returns HL_OK (0) or a negative code.
 * hl_last_error() gives a human-readable message for the last failure on a
 * handle.  After HL_ECUDA or HL_ETIMEOUT a handle is poisoned: later calls
 * return HL_ESTATE until hl_destroy.  A handle must not be used from two
 * host threads at once; distinct handles are independent.
 *
 * Streams: all device work of a handle is issued on its stream (the legacy
 * default stream unless hl_set_stream was called).  hl_step is stream-ordered
 * and does not synchronise; hl_get_fields and hl_sync do.
 *
 * Ownership: the library never frees memory it did not allocate.  Device
 * buffers bound with hl_bind_device stay owned by the caller and must outlive
 * the handle (or the next hl_bind_device call).
 */
#ifndef HL_H
#define HL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hl_solver hl_solver;

enum {
    HL_OK = 0,
    HL_EINVAL = -1,      /* invalid argument                                   */
    HL_ENOMEM = -2,      /* device or host allocation failed                   */
    HL_ECUDA = -3,       /* a CUDA call failed (handle poisoned)               */
    HL_ETIMEOUT = -4,    /* a bounded device wait expired (handle poisoned):
                            the tensor-core kernels wait on their own MMAs
                            with an iteration limit; no kernel waits on
                            another launch or on the host                    */
    HL_ENONFINITE = -5,  /* a NaN or Inf appeared in the updated node data     */
    HL_ESTATE = -6       /* call not valid in the handle's state               */
};

/* Arithmetic modes for hl_set_precision.  The node data are binary64 and
 * every increment is added to them in binary64 in all modes. */
enum {
    HL_FP64 = 0,         /* every operation in IEEE binary64                   */
    HL_FP32 = 1,         /* interpolation + evolution contraction on the FP32
                            pipe: data and operator rounded to binary32, FP32
                            accumulation                                     */
    HL_FP32_COMP = 2,    /* as HL_FP32 with a split-precision correction:
                            data and operator as binary32 hi + lo pairs and
                            float-float arithmetic throughout (error-free
                            TwoSum / TwoProduct), about 48 significant bits  */
    HL_TC_SPLIT = 3      /* dim = 2 (m <= 3) and dim = 3 (m = 2, one shot):
                            the contraction as exact FP16 digit products on
                            the fifth-generation tensor cores (tcgen05.mma,
                            FP32 accumulators in tensor memory): the binary64
                            partner data (scaled by the largest power of two
                            of the whole field, or of a 128-node tile's
                            region for a batch of 2D shots) and the
                            operator cut into 6
                            base-256 digits; the digit pairs of the 7
                            leading levels are summed, each level exactly,
                            then in float-float; about 46 bits below that
                            maximum.  One grid allocates digit planes of
                            both fields (1.5x the state's size)             */
};

/*
 * hl_create -- allocate a solver for the periodic unit box.
 *   dim     : 1, 2 or 3 (Section 2 for dim = 1; Section 5 for the tensor grids).
 *   m       : Hermite order, 0 <= m <= 6 (the paper runs up to m = 6 in
 *             Section 5.3); dim = 3 allows m <= 3.
 *   n_cells : dim entries, nodes per axis per grid, each >= 2.
 *   dt      : time step, 0 < dt < min_k h_k.  The update is the exact
 *             evolution of the interpolant only while c*dt/dx < 1 (Section 3,
 *             the remark before eq. ph1evolve); C_CFL = dt/min h_k = 0.9 is
 *             the paper's usual choice (Section 4, Tables 1-5).
 *   out     : receives the handle (set to NULL on failure).
 * Returns HL_EINVAL on bad arguments (before any CUDA call), HL_ENOMEM or
 * HL_ECUDA if device set-up fails.  The state is zero after creation.
 */
int hl_create(int dim, int m, const int64_t *n_cells, double dt, hl_solver **out);

/*
 * hl_create_batch -- one handle for n_shots independent grids of the same
 * dim and m, stepped together (every launch covers all shots; hl_step is
 * captured as one CUDA graph by default).
 *   n_shots : 1..256; batched handles allow m <= 3.
 *   n_cells : n_shots*dim entries, shot-major.
 *   dt      : n_shots time steps (each below that shot's min h).
 * Host layout of a batch: the single-grid layouts of the shots concatenated
 * in shot order (p blocks, then separately u blocks); the device layout is
 * the concatenation of each shot's slot-major blocks.  hl_get_fields reports
 * the times of shot 0; shot s is at steps*dt[s] (see hl_info).
 * Validation and error codes as hl_create.
 */
int hl_create_batch(int dim, int m, int n_shots, const int64_t *n_cells, const double *dt, hl_solver **out);

/*
 * hl_create_spacing -- hl_create for a periodic grid whose node spacing is
 * not 1/n_cells[k]: n_cells[k] nodes spaced h_k = 1/inv_h[k] apart, period
 * n_cells[k]/inv_h[k] along axis k.  The update's Courant parameter is
 * lam_k = dt*inv_h[k]/2 = dt/(2 h_k) (Section 2: the interpolant lives on a
 * cell of width h and is evolved over dt/2), so hl_create(dim, m, n, dt) is
 * hl_create_spacing with inv_h = n, bit for bit.
 *   inv_h : dim entries, finite and > 0.
 *   dt    : 0 < dt < min_k h_k.
 * Its use is the slab of a larger grid: a process that owns L planes of an
 * axis of N nodes creates L + 2 planes with inv_h = N along that axis, the
 * outer two being ghost copies of its neighbours' edge planes, refreshed
 * before every step.  Point sources and the learned-correction calls assume
 * the unit box and reject a handle whose inv_h differs from n_cells
 * (HL_EINVAL).  Other validation and error codes as hl_create.
 */
int hl_create_spacing(int dim, int m, const int64_t *n_cells, const double *inv_h, double dt, hl_solver **out);

/*
 * hl_set_initial -- copy host initial data (host layout) to the device.
 *   p : prod(n_cells)*nq doubles, p at t = 0.
 *   u : dim*prod(n_cells)*nq doubles, u at t = dt/2.
 * Resets the step counter to 0.  Synchronous with respect to the host
 * buffers (they may be reused on return).  Pinned host memory is fastest.
 */
int hl_set_initial(hl_solver *h, const double *p, const double *u);

/*
 * hl_set_initial_device / hl_get_fields_device -- as hl_set_initial /
 * hl_get_fields but with DEVICE pointers in the host layout; stream-ordered,
 * no host synchronisation.
 */
int hl_set_initial_device(hl_solver *h, const double *p_dev, const double *u_dev);
int hl_get_fields_device(hl_solver *h, double *p_dev, double *u_dev);

/*
 * hl_step -- advance n_steps >= 0 full steps (p-half then u-half each;
 * Section 6 counts one such p-and-v pass as an iteration).  Stream-ordered;
 * returns after enqueueing.  A NaN/Inf produced by the update is reported by
 * the next hl_sync / hl_get_fields as HL_ENONFINITE.
 */
int hl_step(hl_solver *h, int64_t n_steps);

/*
 * hl_get_fields -- copy the state to host buffers (host layout) and
 * synchronise.  Any pointer may be NULL to skip that output.
 *   t_p receives n*dt (time of p), t_u receives (n + 1/2)*dt (time of u).
 * Returns HL_ENONFINITE if any update since the last check produced a
 * non-finite value (the data are still copied).
 */
int hl_get_fields(hl_solver *h, double *p, double *u, double *t_p, double *t_u);

/*
 * hl_sync -- wait for the handle's stream and report the device status
 * (HL_OK, HL_ENONFINITE, or HL_ECUDA).  Clears the non-finite flag.
 */
int hl_sync(hl_solver *h);

/* hl_destroy -- release everything the library allocated for h (NULL is a no-op). */
void hl_destroy(hl_solver *h);

/* hl_last_error -- message for the last failure on h (never NULL; "" if none). */
const char *hl_last_error(const hl_solver *h);

/*
 * hl_set_stream -- issue the handle's device work on cuda_stream (a
 * cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream); NULL selects
 * the legacy default stream.  Synchronises the previous stream first.
 */
int hl_set_stream(hl_solver *h, void *cuda_stream);

/*
 * hl_bind_device -- make the solver operate in place on caller-owned device
 * buffers in the DEVICE layout (slot-major): p_dev[q][node] (nq*nnode
 * doubles) and u_dev[comp][q][node] (dim*nq*nnode doubles), each 16-byte
 * aligned.  The current contents of the bound buffers become the state
 * (no copy); the step counter is kept.  Passing NULL for both returns to
 * library-owned buffers (state zeroed).
 */
int hl_bind_device(hl_solver *h, double *p_dev, double *u_dev);

/*
 * hl_set_source -- add a point source to the pressure equation,
 *     p_t + div u = amp * R(t) * g(x),
 *     R(t) = (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2), t0 = 1.2/f0
 *     (a Ricker wavelet of peak frequency f0),
 *     g(x) = exp(-|x - x0|^2 / (2 sigma^2)) (nearest periodic image of x0),
 * injected after every p-half by the midpoint rule:
 *     p~_a += dt * amp * R((n + 1/2) dt) * g~_a  (g~ = exact scaled derivatives).
 * The paper forces its manufactured-solution experiments with a source
 * z(x,t) in the pressure equation (Section 4, eq. waveEq1D) but states no
 * time discretisation; this midpoint rule is second order in time.  g~ is
 * evaluated on the nodes within 10 sigma of x0 per axis (g < e^-50 outside).
 *   x0 : dim coordinates in [0,1); sigma > 0; f0 > 0; amp = 0 removes the source.
 * The source time of step n is taken from the handle's step counter.
 */
int hl_set_source(hl_solver *h, const double *x0, double sigma, double f0, double amp);

/*
 * hl_set_sources -- per-shot point sources for a batched handle (arrays of
 * n_shots entries; x0 has n_shots*dim).  Shots with amp[s] = 0 get none.
 * Same source model and injection as hl_set_source.
 */
int hl_set_sources(hl_solver *h, const double *x0, const double *sigma, const double *f0, const double *amp);

/*
 * hl_set_wave_speed -- a spatially varying wave speed (Section 4.2), dim = 1:
 *     p_t + c^2(x) u_x = 0,   u_t + p_x = 0.
 * c2_primal and c2_dual hold, for every primal and every dual node, the scaled
 * Taylor coefficients h^i/i! d^i c^2 (i = 0..2m+1) of c^2 at that node: host
 * arrays [node][2m+2] (the paper's local expansion of the coefficient, with
 * the printed h!/i! read as h^i/i!).  Each half-step then runs the
 * Cauchy-Kowalevsky recurrence with these polynomials kept to degree 2m+1
 * and sums the odd temporal terms to order 2m+1.  Both NULL restores unit
 * speed.  Requires one grid, HL_FP64, c^2 > 0 and max c * dt < h at the node
 * values (HL_EINVAL otherwise); takes effect at the next hl_step.
 */
int hl_set_wave_speed(hl_solver *h, const double *c2_primal, const double *c2_dual);

/* Wall kinds for hl_set_walls. */
enum {
    HL_WALL_PERIODIC = 0,   /* no wall along the axis                              */
    HL_WALL_DIRICHLET = 1,  /* p = 0 on the walls (pressure release; a perfect
                               conductor for E_z in Maxwell TM form): p odd across
                               the wall, the normal velocity even, tangential odd */
    HL_WALL_NEUMANN = 2     /* d_n p = 0 (rigid): p even, normal velocity odd      */
};

/*
 * hl_set_walls -- reflecting walls by ghost mirroring (Section 5.2, eq.
 * Boundary and the mirroring that follows it; Section 5.3 runs Maxwell's TM
 * equations, this system with p = E_z and u = (-H_y, H_x), through the same
 * walls).  kinds: dim entries (HL_WALL_*), NULL removes the walls.
 * The handle's grid must be laid out for walls: along a walled axis of N
 * cells of width h it has N + 2 planes spaced h (hl_create_spacing): plane 0
 * is an unused primal plane and a dual ghost, planes 1 .. N+1 the primal
 * nodes 0 .. N (both walls included), planes 1 .. N the dual nodes 0 .. N-1,
 * plane N+1 the second dual ghost.  Before every p-half hl_step fills, axis
 * by axis, the dual ghosts with the mirror images of dual planes 1 and N
 * (slot a times s (-1)^(a_k), s the parity of the velocity component across
 * the wall) and zeroes primal plane 0, on the handle's stream (no host
 * synchronisation; captured with the steps in graph mode).  One grid, HL_FP64
 * or HL_TC_SPLIT, at least 4 planes along walled axes; HL_EINVAL otherwise.
 */
int hl_set_walls(hl_solver *h, const int *kinds);

/*
 * hl_autotune -- time every tile shape (HL_OPT_TILE) on scratch copies of the
 * state (the solution is not advanced), steps_per_trial steps each after one
 * warm-up step, and keep the fastest.  best_tile receives its index and
 * ms_per_tile[HL_NUM_TILES] (may be NULL) the milliseconds per step of each
 * shape (-1 for shapes not tried).  Allocates scratch equal to the state size.
 */
int hl_autotune(hl_solver *h, int64_t steps_per_trial, int *best_tile, double *ms_per_tile);

/*
 * hl_set_precision -- select the arithmetic mode (HL_FP64, HL_FP32,
 * HL_FP32_COMP, HL_TC_SPLIT).  The mixed modes need m <= 3 (m <= 2 in 3D;
 * HL_TC_SPLIT: dim 2 or 3, in 3D m = 2 and a single shot) and, on a batch,
 * the same dt/h on every shot; they return HL_EINVAL otherwise (HL_ENOMEM
 * when the 3D digit planes do not fit).  Takes effect at the next hl_step.
 */
int hl_set_precision(hl_solver *h, int mode);

/* Options for hl_set_option. */
enum {
    HL_OPT_KERNEL_PATH = 1,  /* 0 = automatic; 1 = one persistent CTA with the
                                whole state in shared memory (tiny grids only);
                                2 = one grid launch per half-step             */
    HL_OPT_TIMING = 2,       /* 1 = bracket every kernel launch with CUDA events
                                on the handle's stream (read by hl_kernel_times);
                                0 = off (default).  Not recorded in graph mode. */
    HL_OPT_GRAPH = 3,        /* 1 = capture each hl_step call (all its launches)
                                as one CUDA graph and launch that; default 1 for
                                batched handles, 0 otherwise                  */
    HL_OPT_TILE = 4,         /* thread-block tile shape index 0..HL_NUM_TILES-1
                                (nodes per block along x and y: 128x1, 256x1,
                                64x2, 32x4, 32x8, 64x4, 16x8, 16x16; then the
                                paired shapes 32x4, 32x8, 64x4, 16x16 whose
                                FP64 kernels give each thread two nodes
                                adjacent along y in both half-steps, and
                                32x8, 64x4 paired in the p-half only; dim = 1
                                folds the tile into x and never pairs);
                                hl_autotune picks one                          */
    HL_OPT_STEP = 5,         /* set the step counter n (>= 0) that places the
                                state in time (p at n dt, u at (n + 1/2) dt) and
                                clocks the point sources; hl_set_initial resets
                                it to 0, so a run resumed from a checkpoint
                                sets it back to the checkpoint's step count    */
    HL_OPT_SPLIT = 6         /* 1 = run each FP64 half-step as the split pair of
                                Section 6 (the comparison of Figs. 5-6 and
                                Table 6): an interpolation kernel stores every
                                node's (2m+2)^dim interpolant coefficients per
                                partner component (sum-factorised, one axis at
                                a time) to a device buffer, an evolution kernel
                                reads them back and sums the Cauchy-Kowalevsky
                                series; 0 = the fused kernels (default).  One
                                grid, m <= 3, HL_FP64, unit speed; allocates
                                dim (2m+2)^dim doubles per node (HL_ENOMEM)   */
};

#define HL_NUM_TILES 14

/*
 * hl_set_option -- set an execution option (see the HL_OPT_* values).
 * Returns HL_EINVAL for an unknown option or value.  Options other than
 * HL_OPT_STEP change how the work is scheduled, never what is computed.
 */
int hl_set_option(hl_solver *h, int option, int64_t value);

/*
 * hl_kernel_times -- durations of the kernel launches recorded while
 * HL_OPT_TIMING was on, since the previous call (which resets them).
 * Synchronises the handle's stream.
 *   ms[3]       : total milliseconds of p-half launches, u-half launches and
 *                 single-CTA whole-run launches (any pointer may be NULL);
 *   launches[3] : the matching launch counts.
 */
int hl_kernel_times(hl_solver *h, double *ms, int64_t *launches);

/*
 * hl_operator_table -- the fused per-node operator the FP64 kernels apply,
 * for inspection (host only, no CUDA call).  out receives dim*nq*nq doubles,
 * entry (i, l, s) at (i*nq + l)*nq + s: the increment of output slot s per
 * unit of the vertex butterfly of input slot l, direction i, with
 * lam[k] = dt/(2 h_k).  It is W_i (H x ... x H) restricted to the all-lower
 * vertex block and negated (Section 2, eqs. interp and final1; Section 3.1.2,
 * eqs. pdup and vdup), composed in double-double and rounded once.
 */
int hl_operator_table(int dim, int m, const double *lam, double *out);

/*
 * hl_tc_tables -- the operator digit tables of the tensor-core split mode
 * (HL_TC_SPLIT, dim = 2), for inspection (host only, no CUDA call).
 *   m      : 0..3;  lam : 2 entries, dt/(2 h_k).
 *   digits : HL_TC_TABLE_ELEMS uint16 (BF16 bit patterns of small integers).
 *            Entry (op, j, s, k) at ((op*6 + j)*16 + s)*136 + k: digit j
 *            (most significant first) of row k of output column s of
 *            operator op.  op 0 is the p-half (rows k = (c*4 + v)*16 + l:
 *            velocity component c, cell vertex v, slot l); ops 1 and 2 are
 *            the u-half for directions 0 and 1 (rows k = v*16 + l of p).
 *            Vertex v has bit k set for the upper vertex along axis k; rows
 *            and columns beyond the (m+1)^2 slots, and k >= 128, are zero.
 *   expo   : HL_TC_EXPO_ELEMS ints, e(op, s) at op*16 + s.
 * The operator entry is (sum_j digit_j 256^(5-j)) 2^(e - 46): the vertex form
 * of the fused operator (the increment of output slot s per unit of the
 * partner's slot l at vertex v), rounded to 46 bits below its column's
 * maximum (an Ozaki-type exact split: every digit product is exact in FP32).
 */
#define HL_TC_TABLE_ELEMS 39168
#define HL_TC_EXPO_ELEMS 48

/*
 * hl_tc_image -- the operator images the tensor-core split kernels load, as
 * they load them (host only, no CUDA call), for inspection.  Entries are the
 * FP16 bit patterns of the balanced base-256 digits of hl_tc_tables' scheme
 * (integers in [-128, 127]); the entry is (sum_j digit_j 256^(5-j)) 2^(e - 46).
 *   dim 2 (m <= 3): HL_TC_IMAGE2_ELEMS entries, p-half then u-half (14336
 *     each): blocks b of [2 chunks][R rows][8 slots], slot l = chunk*8 + k;
 *     p-half b = c*4 + v, R = 112, row n = j*16 + s; u-half b = v, R = 224,
 *     row n = j*32 + i*16 + s (direction i); expo HL_TC_EXPO_ELEMS ints as in
 *     hl_tc_tables.
 *   dim 3 (m = 2): HL_TC_IMAGE3_ELEMS entries, p-half then u-half (172032
 *     each): 12 units u = (i*2 + vz)*2 + kh (i: velocity component for the
 *     p-half, direction for the u-half; vz the vertex's z bit; kh the half of
 *     the 32 padded slots), each 4 vertex blocks vx + 2 vy of [2 chunks][224
 *     rows n = j*32 + s][8 slots], slot l = kh*16 + chunk*8 + k; expo
 *     HL_TC_EXPO3_ELEMS ints, e(op, s) at op*32 + s (op 0 the p-half, 1 + i
 *     the u-half's direction i).
 * Digit row block j = 6 and every slot beyond the node's (m+1)^dim are zero.
 * lam[k] = dt/(2 h_k).  Returns HL_EINVAL for other (dim, m) or short buffers.
 */
#define HL_TC_IMAGE2_ELEMS 28672
#define HL_TC_IMAGE3_ELEMS 344064
#define HL_TC_EXPO3_ELEMS 128
int hl_tc_image(int dim, int m, const double *lam, uint16_t *image, int64_t image_elems, int *expo,
                int64_t expo_elems);
int hl_tc_tables(int m, const double *lam, uint16_t *digits, int *expo);

/*
 * hl_op_counts -- floating-point work of the FP64 kernels per node and full
 * step for (dim, m): multiply-adds (one multiply-add = 2 flops) and plain
 * additions of the vertex butterflies.  Used for roofline accounting.
 */
int hl_op_counts(int dim, int m, double *fma_per_node_step, double *add_per_node_step);

/*
 * hl_info -- sizes of a handle: nnode (nodes per grid, summed over the shots
 * of a batch), nq ((m+1)^dim) and the number of completed steps.  Any pointer may be NULL.
 */
int hl_info(const hl_solver *h, int64_t *nnode, int64_t *nq, int64_t *steps);

/*
 * hl_step_noalloc -- advance n_steps FP64 steps of one periodic grid held in
 * caller-owned device buffers (device layout, as hl_bind_device), with no
 * device allocation at all.  For callers that cannot call cudaMalloc: code
 * living inside a device memory budget owned by another application,
 * real-time loops that forbid allocation after start-up, or hosts whose
 * allocator is locked while they run.  The paper has no counterpart; this is
 * a deployment variant of hl_step.
 *   dim, m, n_cells, dt : as hl_create; p_dev, u_dev : the state, updated in
 *   place; cuda_stream : stream to run on (NULL = legacy default stream).
 * The kernels' scratch (status word, grid descriptor and, when it does not fit
 * the kernel parameter bank, the operator table) lives in one file-scope
 * static device array of HL_NOALLOC_SCRATCH_BYTES, held by every GPU that
 * loads the library until the process exits.  Operators larger than that
 * (3D m = 3) are rejected with HL_EINVAL.  The first call on a device does a
 * host-side set-up step: it looks up the array's device address on that device
 * (cudaGetSymbolAddress, with the device current); that first call should come
 * before any stream capture.  Every call ends by copying the status word back
 * to a host variable and synchronising the stream.
 * Every call shares the array and clears the status word it uses: calls that
 * overlap on the GPU (other streams, other host threads) race on it.
 * p_dev and u_dev must be device memory of the current device (checked with
 * cudaPointerGetAttributes, which allocates nothing; HL_EINVAL otherwise).
 * Returns HL_OK, HL_ENONFINITE, HL_EINVAL or HL_ECUDA; hl_last_error(NULL)
 * describes a failure.  Host memory is used only to build the operator table.
 */
#define HL_NOALLOC_SCRATCH_BYTES 65536
int hl_step_noalloc(int dim, int m, const int64_t *n_cells, double dt, double *p_dev, double *u_dev,
                    int64_t n_steps, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Modified Hermite-leapfrog scheme (Section 4.3; eqs. hy1, hy2, lfw1, lfw2 and
 * the pressure-velocity experiment of Table 4), 1D: p_t + u_x = 0, u_t + p_x = 0
 * on the periodic unit interval, n_cells nodes per grid, h = 1/n_cells.
 * Both fields live on both grids: primal nodes j h hold (p, u) at t = n dt,
 * dual nodes (j + 1/2) h hold (p, u) at t = (n + 1/2) dt.  A step updates the
 * primal grid from the dual grid's interpolants (the cell around primal node j
 * has dual nodes j - 1 and j as vertices), then the dual grid from the primal
 * one (vertices: primal nodes j and j + 1).  Even derivative slots take the
 * difference of the forward and backward temporal Taylor expansions about the
 * midpoint (eq. hy1), odd slots their sum (eq. lfw2), with the full series of
 * the degree-2m+1 interpolant; the paper reports uniform order 2m+2.
 * Host layout of each of the four arrays: f[node][q], q = 0..m (scaled
 * derivatives h^q/q! d^q f), node x-fastest.  Device layout is private.
 * Errors as the hl_* calls; hl_mod_last_error(NULL) describes a failed create.
 */
typedef struct hl_mod hl_mod;

/* hl_mod_create -- 0 <= m <= 6, n_cells >= 2, 0 < dt < 1/n_cells; state zero. */
int hl_mod_create(int m, int64_t n_cells, double dt, hl_mod **out);
void hl_mod_destroy(hl_mod *h);
const char *hl_mod_last_error(const hl_mod *h);
/* hl_mod_set_stream -- as hl_set_stream. */
int hl_mod_set_stream(hl_mod *h, void *cuda_stream);
/*
 * hl_mod_set_initial -- copy host data: pp, up (primal grid, t = 0) and pd, ud
 * (dual grid, t = dt/2), each n_cells*(m+1) doubles; resets the step counter.
 * Synchronous with respect to the host buffers.
 */
int hl_mod_set_initial(hl_mod *h, const double *pp, const double *up, const double *pd, const double *ud);
/* hl_mod_step -- n_steps >= 0 full steps, stream-ordered (no synchronisation). */
int hl_mod_step(hl_mod *h, int64_t n_steps);
/*
 * hl_mod_get_fields -- copy the state to host buffers (NULL skips one) and
 * synchronise; HL_ENONFINITE if an update since the last check produced a
 * NaN or Inf (the data are still copied).
 */
int hl_mod_get_fields(hl_mod *h, double *pp, double *up, double *pd, double *ud);
/* hl_mod_info -- completed steps and the times of the primal and dual data. */
int hl_mod_info(const hl_mod *h, int64_t *steps, double *t_primal, double *t_dual);

/* ------------------------------------------------------------------------
 * Learned coarse-grid correction (not in the paper).  A per-node multilayer
 * perceptron over a coarse 2D m = 3 solution predicts, for every primal node,
 * corrections to its 16 scaled p values; it is trained on fine-grid solutions
 * produced by this solver.  Features of coarse primal node J (feat_scale times
 * the node data, t_feature as given, zero padded):
 *     p at the 3x3 primal nodes J + {-1,0,1}^2 (y offset outer)      144
 *     u then v at the cell vertices, dual nodes J + {-1,0}^2          128
 *     t_feature                                                        1
 * Network: 288 -> 128 (ReLU) -> 128 (ReLU) -> 16, every product on the tensor
 * cores with BF16 operands and FP32 accumulation, FP32 master weights and Adam
 * moments.  Loss: mean of (y - target)^2 over rows and outputs.  Parameter
 * block (floats): W1[288][128], b1[128], W2[128][128], b2[128], W3[128][16],
 * b3[16].
 * Every hl_mlp call runs on the handle's stream (hl_mlp_set_stream); device
 * buffers are row-major float, one row per node.
 */
#define HL_MLP_IN 288
#define HL_MLP_HIDDEN 128
#define HL_MLP_OUT 16
#define HL_MLP_NPARAMS 55568

typedef struct hl_mlp hl_mlp;

/* hl_mlp_create -- allocate a network with He-initialised weights (seeded). */
int hl_mlp_create(uint64_t seed, hl_mlp **out);
void hl_mlp_destroy(hl_mlp *mlp);
const char *hl_mlp_last_error(const hl_mlp *mlp);
int hl_mlp_set_stream(hl_mlp *mlp, void *cuda_stream);

/*
 * hl_mlp_params -- host copies of the parameters: get_params/get_grads
 * receive HL_MLP_NPARAMS floats (the gradients of the last hl_mlp_loss_grad);
 * set_params replaces the weights and resets Adam.  Any pointer may be NULL.
 * Synchronises the handle's stream; HL_ETIMEOUT if an earlier hl_mlp_forward
 * reported an expired tensor-core wait.
 */
int hl_mlp_params(hl_mlp *mlp, float *get_params, const float *set_params, float *get_grads);

/*
 * hl_mlp_forward -- Y_dev[rows][16] = network(X_dev[rows][288]), on the
 * network's stream.  With X_dev and Y_dev 16-byte aligned, one tcgen05 kernel
 * runs all three layers per 128-row tile with the activations on chip (FP32
 * accumulators in tensor memory); otherwise the per-layer GEMMs of
 * hl_mlp_loss_grad run.  Both round the operands to BF16 and accumulate in
 * FP32.  A bounded tensor-core wait that expires is reported as HL_ETIMEOUT by
 * the next hl_mlp_params call, or hl_mlp_loss_grad call that returns a loss
 * (the handle is then poisoned).
 */
int hl_mlp_forward(hl_mlp *mlp, const float *X_dev, int rows, float *Y_dev);

/*
 * hl_mlp_loss_grad -- forward (as hl_mlp_forward; the tensor-core kernel
 * also keeps the FP32 activations for the backward pass), loss against
 * T_dev[rows][16] and the full gradient (overwrites the previous one) by
 * per-layer GEMMs.  loss (host, may be NULL) receives the mean squared error;
 * passing it synchronises the stream and reports an expired tensor-core wait
 * (HL_ETIMEOUT).
 */
int hl_mlp_loss_grad(hl_mlp *mlp, const float *X_dev, const float *T_dev, int rows, double *loss);

/*
 * hl_mlp_sample -- draw a training minibatch on the device: row i of draw
 * `step` copies pool row splitmix64(seed + (step*rows + i + 1) * 0x9e3779b97f4a7c15)
 * mod pool_rows (SplitMix64, Steele, Lea and Flood 2014) from X_pool[pool_rows][288]
 * (and T_pool[pool_rows][16], may be NULL) into X_dev[rows][288] (and T_dev),
 * on the network's stream.  The paper has no counterpart: this is training
 * plumbing for the learned correction, so that a training loop needs no host
 * round trip.  All buffers are device memory owned by the caller.
 */
int hl_mlp_sample(hl_mlp *mlp, const float *X_pool, const float *T_pool, int64_t pool_rows, int rows, uint64_t seed,
                  uint64_t step, float *X_dev, float *T_dev);

/* hl_mlp_adam_step -- one Adam update (beta1 0.9, beta2 0.999, eps 1e-8) with the current gradient. */
int hl_mlp_adam_step(hl_mlp *mlp, float lr);

/*
 * hl_mlp_grad_buffer -- *grads_dev receives the device address of the
 * network's gradient: HL_MLP_NPARAMS floats (the parameter layout of
 * hl_mlp_params), owned by the network and valid until hl_mlp_destroy, written
 * by hl_mlp_loss_grad (the gradient of the mean squared error over its rows)
 * and read by hl_mlp_adam_step, both on the network's stream.  Data-parallel
 * training reduces it in place between those two calls, on that stream: with
 * equal rows per rank, the mean over the ranks is the gradient of the mean loss
 * over all their rows.  No CUDA call; HL_EINVAL for NULL arguments.
 */
int hl_mlp_grad_buffer(hl_mlp *mlp, float **grads_dev);

/*
 * hl_features -- X_dev[rows][288] for the coarse primal nodes nodes_dev[rows]
 * (device int array; NULL = nodes 0..rows-1) of a single 2D m = 3 grid, on the
 * solver's stream.  Nodes outside the grid give zero rows.
 */
int hl_features(const hl_solver *coarse, const int *nodes_dev, int rows, float feat_scale, float t_feature,
                float *X_dev);

/*
 * hl_targets -- T_dev[rows][16] = (fine p restricted to the coarse node -
 * coarse p) / out_scale.  The fine grid has ratio times the coarse nodes per
 * axis; coarse primal node J is fine primal node ratio*J and slot a of the
 * fine data is scaled by ratio^|a| (h^|a| in the scaled derivatives).  Both
 * solvers must hold data at the same time.  On the coarse solver's stream.
 */
int hl_targets(const hl_solver *fine, int ratio, const hl_solver *coarse, const int *nodes_dev, int rows,
               double out_scale, float *T_dev);

/*
 * hl_apply_correction -- p~(J) += out_scale * network(features(J)) at every
 * primal node of the coarse solver (the addition in FP64; the network as
 * hl_mlp_forward).  Uses workspace owned by the network handle.  An expired
 * tensor-core wait is reported by the solver's next hl_sync as HL_ETIMEOUT.
 */
int hl_apply_correction(hl_solver *coarse, hl_mlp *mlp, float feat_scale, float t_feature, double out_scale);

/*
 * hl_set_correction -- apply the learned correction inside the stepping loop:
 * after every every_k_steps-th step of the handle's step count, hl_step runs
 * on the handle's stream (no host synchronisation, CUDA-graph capturable)
 *     y = network(features(J)) at every primal node J     (as hl_apply_correction)
 *     p~(J) += out_scale * y                               (in FP64)
 * unless the plain solver judges it unsafe.  Fallback rule: the correction is
 * skipped (the plain step stands) when
 *     sum_J,q (out_scale y)^2  >  max_ratio^2 * sum_J,q (p~ - p~_before)^2,
 * p~_before being p before the last plain step: a correction larger than
 * max_ratio times that step's own change (or a non-finite one) is not taken.
 * The paper has no learned correction; this is the run-time use of the
 * coarse-grid correction trained by the hl_mlp_* calls, on a single 2D m = 3
 * unit-box grid in HL_FP64.  mlp == NULL removes the correction; the network
 * handle must outlive its use and must not run other work concurrently (its
 * workspace is used).  Allocates p-sized scratch once (HL_ENOMEM on failure).
 */
int hl_set_correction(hl_solver *h, hl_mlp *mlp, int every_k_steps, float feat_scale, float t_feature,
                      double out_scale, double max_ratio);

/* hl_correction_stats -- corrections applied and skipped so far (synchronises). */
int hl_correction_stats(hl_solver *h, int64_t *applied, int64_t *skipped);

#ifdef __cplusplus
}
#endif

#endif /* HL_H */

/*
 * cteno.h -- C ABI of the GB300 (sm_103a) CTENO / CTENOZ finite-volume library.
 *
 * The library advances the compressible Euler equations (paper eq. 1) on triangle (2D) and
 * tetrahedron (3D) meshes with the semi-discretisation of eq. 2: a per-cell high-order
 * reconstruction (Sec. 2.1-2.6: reference-space least squares, eqs. 5-12; smoothness indicators,
 * eq. 15; CWENO optimal-polynomial split, eqs. 16-18; CTENO selection, Alg. 1, or CTENOZ
 * selection, Alg. 2), the HLLC flux at face Gauss points (Sec. 2.7, eqs. 24-29), and the
 * explicit third-order Runge-Kutta update (Sec. 2, after eq. 2). Several independent meshes can
 * share one context; each RK stage advances all of them in the same kernel launches.
 *
 * Conventions, for every entry point:
 *   - Return 0 on success or a negative CTENO_ERR_* code. The message of the last failure is
 *     cteno_last_error(ctx). A context whose device state reported a fault (a non-finite state,
 *     or a bounded wait for a bulk copy that ran out) returns CTENO_ERR_DEVICE from every later
 *     synchronising call. Every index the kernels gather with (stencil members, face neighbours,
 *     staging lists) is checked on the host when cteno_lsq_build uploads it.
 *   - Input arrays are copied; the library never keeps a caller's pointer. Output arrays are
 *     allocated by the caller.
 *   - Host pointers are plain host memory; "device" pointers are CUDA device (or managed)
 *     memory of the context's device.
 *   - Work is enqueued on the stream passed to cteno_create (borrowed, never destroyed) and the
 *     call returns without synchronising, except the cteno_get_* calls that write host memory,
 *     cteno_sync and cteno_lsq_build, which synchronise that stream.
 *   - State layout at the boundary: conserved cell means U[v][c], variable-major, v = 0..d+1
 *     (rho, rho u, rho v[, rho w], E), c in the caller's original cell numbering of that mesh.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef CTENO_H
#define CTENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CTENO_OK = 0,
  CTENO_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, bad parameter) */
  CTENO_ERR_STATE = -2,    /* call out of order (e.g. rk_stage before lsq_build) */
  CTENO_ERR_MESH = -3,     /* degenerate cell, non-manifold face, or bad connectivity */
  CTENO_ERR_STENCIL = -4,  /* a cell cannot gather M = 2K stencil cells */
  CTENO_ERR_RANK = -5,     /* a central least-squares matrix is rank deficient */
  CTENO_ERR_CUDA = -6,     /* a CUDA runtime call failed (message has the CUDA error) */
  CTENO_ERR_DEVICE = -7,   /* a kernel reported a fault in its error word */
  CTENO_ERR_NOMEM = -8     /* host or device allocation failed */
};

enum { CTENO_SCHEME_CTENO = 0, CTENO_SCHEME_CTENOZ = 1, CTENO_SCHEME_CWENO = 2, CTENO_SCHEME_TENO = 3 };
enum { CTENO_FP64 = 0, CTENO_MIXED = 1 };
/* Boundary faces of a mesh: transmissive (the outside state is the cell mean) or reflective walls
 * (the outside state at each Gauss point is the mirror image of the reconstructed inside state,
 * (rho, m - 2 (m.n) n, E); the paper's Sec. 3.3 and 3.4 run walls without printing their
 * treatment). Periodic directions have no boundary faces. */
enum {
  CTENO_BOUNDARY_TRANSMISSIVE = 0,
  CTENO_BOUNDARY_WALL = 1,
  CTENO_BOUNDARY_STATE_A = 2,  /* the outside state is the fixed state A (inflow, post-shock) */
  CTENO_BOUNDARY_SHOCK_AB = 3  /* 2D: state A where the moving shock line x = xs0 + sy y + vs t has
                                  passed the face midpoint (xs0 + sy y_mid + vs t > x_mid), else B;
                                  t is the stage's time (cteno_set_time / cteno_get_time) */
};

/* Scheme parameters (paper notation). */
typedef struct {
  int dim;              /* d = 2 (triangles) or 3 (tetrahedra) */
  int degree;           /* r: central polynomial degree, order r+1 (Sec. 2.1); 2 or 3, and in 2D
                           also 4 to 6 (CTENO5-7, Sec. 2.3 and Fig. 1: directional stencils of
                           degree 2 with at most 10 members, (r+2)/2 Gauss points per edge; the
                           reconstruction runs the variable-per-lane schedule only) */
  int scheme;           /* CTENO_SCHEME_CTENO (Alg. 1) or CTENO_SCHEME_CTENOZ (Alg. 2); for
                           comparison in the same kernels, CTENO_SCHEME_CWENO (Sec. 2.3: every
                           stencil with the weights of eq. 14, b = 4, on the CWENO split p_1) and
                           CTENO_SCHEME_TENO (Sec. 2.4: the cut-off of eqs. 19-23 without linear
                           coefficients, on the central least-squares polynomial itself) */
  int precision;        /* CTENO_FP64: all arithmetic in FP64. CTENO_MIXED: reconstruction and
                           flux in FP32; geometry, least-squares build, residual accumulation and
                           the RK update in FP64 */
  int lam_gamma;        /* 1: scale-separation measure gamma_s carries the linear coefficient
                           lambda_s of eq. 18 (default, reproduces Tables 1-3); 0: as printed in
                           eq. 19 / Alg. 1-2 */
  int positivity_guard; /* 1: a cell whose face state has rho <= 0 or p <= 0 uses its cell mean
                           at all its face points for that stage (not in the paper) */
  int ctenoz_form;      /* CTENOZ smoothness measure (Sec. 2.6, Alg. 2). 0: as printed,
                           tau = (sum_{s>=2} |SI_s - SI_1| / (s_t - 1))^6, gamma_s = 1 + tau/(SI_s + eps).
                           1: the WENO-Z arrangement, tau = sum_{s>=2} |SI_s - SI_1| / (s_t - 1),
                           gamma_s = 1 + (tau/(SI_s + eps))^6 (a reading; scale invariant) */
  int characteristic;   /* 0: reconstruct the conserved variables, each selected independently.
                           1: reconstruct characteristic variables (Sec. 2.2, 3.2): for each face,
                           W = L U with L the left eigenvectors of the Euler flux Jacobian in the
                           face's outward normal direction at the cell's mean state; every field
                           selected independently; the face's Gauss-point values transformed back
                           with R = L^-1. Reconstruction schedule 1024 + b only */
  int rk;               /* explicit Runge-Kutta step (Sec. 2, "3rd- or 4th-order"): 3 = SSP-RK3
                           (Shu-Osher form, 3 stages), 4 = the classical RK4 (4 stages, one more
                           FP64 state array); cteno_run replays all stages of a step */
  double C_T;           /* cut-off of eq. 23 (paper: 1e-6) */
  double lambda1p;      /* lambda_1' of eq. 18 (paper: 1e4 or 1e15) */
  double eps;           /* epsilon of eqs. 19 and CTENOZ (not given by the paper; default 1e-24,
                           above the rounding floor of the smoothness indicators of both paths for
                           |U| up to ~100, so that no selection depends on rounding; the printed
                           CTENOZ measure drops the central stencil only where tau/eps exceeds
                           about lambda_1'/C_T, so eps also sets its detection threshold) */
  double cfl;           /* Courant number of the time step rule (cteno_run) */
  double gamma;         /* ratio of specific heats (1.4) */
} cteno_params;

typedef struct cteno_ctx cteno_ctx;

/* Fill *p with the defaults: d = 2, r = 2, CTENO, FP64, lam_gamma 1, guard 1, ctenoz_form 0,
 * characteristic 0, rk 3,
 * C_T = 1e-6, lambda_1' = 1e15, eps = 1e-24, CFL 0.5, gamma 1.4. */
void cteno_default_params(cteno_params *p);

/* Create a context on the current CUDA device. `cuda_stream` is a cudaStream_t (may be NULL for
 * the legacy default stream); it is borrowed for the life of the context. The stage kernels use
 * programmatic dependent launch (each kernel is launched as the previous one's blocks exit and
 * waits for its results on the GPU); the environment variable CTENO_PDL=0, read here, launches
 * them plainly instead. CTENO_ZEROCOPY=0 makes the batch-wide state calls stage page-locked host
 * buffers through device memory as well (by default the kernels access them directly, measured
 * faster: 2252 against 2053 Mcell-RK-stage/s end to end on the 131k-cell shock tube). */
int cteno_create(cteno_ctx **out, const cteno_params *p, void *cuda_stream);

/* Append one mesh to the context (Sec. 2: the physical domain as triangles / tetrahedra).
 *   nverts, xyz        : host, xyz[nverts][dim] vertex coordinates (copied).
 *   ncells, cell_verts : host, cell_verts[ncells][dim+1] vertex ids (any orientation; copied).
 *   period             : host, period[dim]; period[j] > 0 makes direction j periodic with that
 *                        length (vertices are stored once and cells unwrap across the box);
 *                        NULL or 0 = bounded.
 *   boundary_kind      : CTENO_BOUNDARY_TRANSMISSIVE, CTENO_BOUNDARY_WALL or
 *                        CTENO_BOUNDARY_STATE_A for every bounded boundary face of this mesh
 *                        (meshes of a batch may differ; cteno_boundary_region refines it).
 *   mesh_id_out        : receives the index of the mesh in the batch.
 * Errors: CTENO_ERR_MESH for degenerate cells or faces shared by more than two cells. Meshes can
 * only be added before cteno_stencil_build. */
int cteno_mesh_build(cteno_ctx *ctx, int64_t nverts, const double *xyz, int64_t ncells,
                     const int32_t *cell_verts, const double *period, int boundary_kind,
                     int32_t *mesh_id_out);

/* Build, on the host, the central stencil of M = 2K cells of every cell (Sec. 2.1, eq. 6; the
 * "SBC" compact stencil) and its directional stencils (Sec. 2.3, Fig. 1), then renumber the cells
 * of each mesh along a Morton curve of their centroids. CTENO_ERR_STENCIL when a cell cannot
 * gather M cells (mesh too small) or a periodic stencil spans too much of the box. */
int cteno_stencil_build(cteno_ctx *ctx);

/* Upload the meshes and build on the GPU, in FP64, the geometry, the basis moments of every
 * stencil in the target cell's reference space (eqs. 5, 7, 10) and their least-squares
 * pseudo-inverses by Householder QR (eq. 12). The mixed path stores them in FP32.
 * CTENO_ERR_RANK when a central matrix is rank deficient. Synchronises. */
int cteno_lsq_build(cteno_ctx *ctx);

/* Set the conserved cell means of one mesh: U[v][c] (layout above), host or device pointer
 * (is_device = 0 / 1). Also computes that mesh's CFL time step of the new state for cteno_run. */
int cteno_set_state(cteno_ctx *ctx, int32_t mesh_id, const double *U, int is_device);

/* Set the conserved cell means of every mesh at once (one copy and one launch for the batch):
 * U holds mesh after mesh, in the order the meshes were added, each mesh's block laid out as
 * for cteno_set_state (nv * ncells values, [v][c] in its own numbering); nv * (total cells)
 * doubles, host or device. Also computes every mesh's CFL time step. A page-locked host buffer
 * is read by the kernel directly, asynchronously: the caller must not modify it until the stream
 * has synchronised (e.g. cteno_sync, or any cteno_get_* call to host memory). Pageable host
 * memory is staged through device memory before the call returns. */
int cteno_set_state_all(cteno_ctx *ctx, const double *U, int is_device);

/* One stage (stage = 0 .. rk - 1) of the Runge-Kutta step (cteno_params.rk), for every mesh. dt:
 * host array of the time step of each mesh (length nmeshes), or NULL: at stage 0 each mesh then
 * takes the CFL step of its current state, dt = CFL min_i |V_i| / sum_f |A_f| (|u_i.n_f| + c_i)
 * (the step cteno_run takes; it is computed by cteno_set_state / cteno_set_state_all and by every
 * last stage), and the later stages keep the step of the last stage 0. Stage 0 stores U^n. */
int cteno_rk_stage(cteno_ctx *ctx, int stage, const double *dt);

/* nsteps full Runge-Kutta steps (SSP-RK3 or RK4, cteno_params.rk), each with dt = CFL * min_i
 * |V_i| / sum_f |A_f| (|u_i.n_f| + c_i) taken per mesh from the state at the start of the step.
 * The stages of a step are captured once into a CUDA graph and replayed. */
int cteno_run(cteno_ctx *ctx, int nsteps);

/* Read the conserved cell means of one mesh into U_out[v][c] (host or device). A host read
 * stages through a device buffer that the context allocates on first use (and grows for a larger
 * mesh); see cteno_get_state_noalloc for a read-back that allocates nothing. */
int cteno_get_state(cteno_ctx *ctx, int32_t mesh_id, double *U_out, int is_device);

/* Read the conserved cell means of every mesh at once into U_out (host or device), laid out as
 * for cteno_set_state_all. A host read synchronises the stream once for the whole batch; a
 * page-locked host buffer is written by the kernel directly. */
int cteno_get_state_all(cteno_ctx *ctx, double *U_out, int is_device);

/* Like cteno_get_state with a host output, but allocating nothing. The paper has no counterpart;
 * this is for callers that cannot allocate device memory at the time they read a state back --
 * for example a program whose memory pool owns all device memory, or code running where
 * cudaMalloc is not allowed. cteno_get_state stages through a device buffer it allocates on first
 * use; this call stages through a 16 MiB array compiled into the library (2^21 doubles), which
 * every GPU that loads the library holds until the process exits.
 *   U_out : host, U_out[v][c] (original numbering), nv * ncells doubles, caller-allocated.
 * Errors: CTENO_ERR_ARG when nv * ncells > 2^21 (the staging area's size); the usual state and
 * mesh checks. The staging array's device address is looked up (cudaGetSymbolAddress) by
 * cteno_lsq_build, on the context's device, once per device; under CUDA's lazy module loading
 * that lookup is also what loads the array onto the device (16 MiB, allocated then), and
 * cteno_lsq_build loads the gather kernel this call launches as well, so the call itself neither
 * allocates nor loads anything. Every call, from any context, shares the one staging array: calls
 * whose work overlaps on the GPU (contexts on different streams at the same time) race and must be
 * serialised by the caller. Nothing in the array needs clearing: each call writes every value it
 * reads back. Synchronises the stream. */
int cteno_get_state_noalloc(cteno_ctx *ctx, int32_t mesh_id, double *U_out);

/* Time step used by the last step of cteno_run for each mesh: host dt_out[nmeshes]. */
int cteno_get_dt(cteno_ctx *ctx, double *dt_out);

/* Enable (1) or disable (0, default) recording of the stencil-selection flags. */
int cteno_record_flags(cteno_ctx *ctx, int enable);

/* Selection flags of the last reconstruction of one mesh, host out[c][v] (original numbering):
 * bit 0 = central stencil kept (delta_1 = 1); bit 1+f = directional stencil of local face f
 * selected (eq. 23 and Alg. 1 / 2). Local faces follow the positively oriented vertex order.
 * With the characteristic reconstruction out[c][f][w]: face f, characteristic field w. */
int cteno_get_flags(cteno_ctx *ctx, int32_t mesh_id, uint8_t *out);

/* Reconstructed face Gauss-point states of the last reconstruction (debug), host
 * out[c][f][q][v], f local face, q canonical point order of the face. FP64 values (the mixed
 * path's FP32 values converted). */
int cteno_get_face_states(cteno_ctx *ctx, int32_t mesh_id, double *out);

/* Host-side stencil of one cell (after cteno_stencil_build, before or after lsq_build):
 * central[M] original cell ids in nearest-first order, dir[(d+1)][nd] positions in `central` of
 * the members of each directional stencil (-1 padded; nd = cteno_info out[8]). Admissibility is known only after
 * cteno_lsq_build; dok may be NULL before it. */
int cteno_get_stencil(cteno_ctx *ctx, int32_t mesh_id, int64_t cell, int32_t *central,
                      int32_t *dir, int32_t *dok);

/* Boundary kinds by region (before cteno_lsq_build): every boundary face of mesh `mesh_id` whose
 * midpoint lies in the axis-aligned box [lo, hi] (host arrays of dim values, inclusive) gets `kind`
 * (CTENO_BOUNDARY_*); later calls override earlier ones, and faces outside every box keep the kind
 * given to cteno_mesh_build. CTENO_ERR_ARG for an unknown kind (or a moving shock in 3D). */
int cteno_boundary_region(cteno_ctx *ctx, int32_t mesh_id, const double *lo, const double *hi, int kind);

/* States A and B (host, nv conserved values each) of the fixed-state and moving-shock kinds, and
 * the moving shock line x = xs0 + sy y + vs t. xs0 and sy enter the face geometry built by
 * cteno_lsq_build, so they must be set before it (CTENO_ERR_STATE after it if they change); A, B
 * and vs may change at any time. */
int cteno_boundary_states(cteno_ctx *ctx, const double *A, const double *B, double xs0, double sy, double vs);

/* Physical time of every mesh (a moving-shock boundary needs it; it starts at 0 and advances by
 * each step's dt, the stages of a step seeing t + c_s dt with c = (0, 1, 1/2) for SSP-RK3 and
 * (0, 1/2, 1/2, 1) for RK4). cteno_set_time sets every mesh's time (a no-op without a moving-shock
 * boundary); cteno_get_time (host t_out[nmeshes]) returns CTENO_ERR_STATE without one. */
int cteno_set_time(cteno_ctx *ctx, double t);
int cteno_get_time(cteno_ctx *ctx, double *t_out);

/* Sizes, out[10]: out[0] = nmeshes, out[1] = total cells, out[2] = M, out[3] = K-1, out[4] = nv,
 * out[5] = faces per cell, out[6] = Gauss points per face, out[7] = cells of mesh `mesh_id`
 * (or 0 if mesh_id < 0), out[8] = members of a directional stencil at most (2d up to degree 3,
 * 10 for degrees 4 to 6), out[9] = selection flags per cell (nv, or (d+1) nv with the
 * characteristic reconstruction). */
int cteno_info(cteno_ctx *ctx, int32_t mesh_id, int64_t *out);

/* Number of cells that fell back to their mean under the positivity guard since the last call,
 * and whether any kernel reported a fault. Synchronises. */
int cteno_sync(cteno_ctx *ctx, int64_t *guard_count);

/* Launch configuration: block sizes of the reconstruction and flux kernels (0 = keep). A negative
 * value -b selects, on the mixed path, the register-capped variant of the kernel (8 resident
 * blocks per SM) with b threads per block, b in {32, 64, 96, 128}. 1024 + b selects the lane
 * schedule with b threads per block (b a multiple of 32 in [32, 256]): for the reconstruction one
 * lane per conserved variable (d+2 lanes per cell), for the flux one lane per face (d+1 lanes per
 * cell). Reconstruction on the mixed path only: 2048 + b / 3072 + b select the thread-per-cell /
 * lane schedule as a persistent kernel that copies each tile's operator records (b cells, or
 * floor(32/(d+2)) cells per warp) into shared memory with bulk copies, two tiles in flight; refused
 * (CTENO_ERR_ARG) when the two stages need more than 200 KiB of shared memory. If a bounded wait for
 * such a copy ever gives up (after 1 s), the kernel stops and the next synchronising call returns
 * CTENO_ERR_DEVICE. 4096 (mixed path) selects that lane schedule with 4 warps whose tiles also copy
 * the states of their distinct stencil members into shared memory (lists built by cteno_lsq_build);
 * 4097 the same with one tile per block and a single stage (half the shared memory); both refused
 * like the staged values when they do not fit. 5120 + w (mixed path, w warps per block, 1..16)
 * selects the streamed lane schedule: every warp walks its own tiles of floor(32/(d+2)) cells and
 * streams their operator records through its own ring of three shared-memory stages, in chunks of
 * 8 (or 4) stencil members per cell, ahead of the arithmetic (bounded waits as above); 5152 + w the
 * same with a two-stage ring; refused when w warps' rings do not fit in the 227 KiB of shared
 * memory of a block. 6144 + w
 * (mixed path, w warps per block, 1..8) selects the streamed thread-per-cell schedule: every warp
 * walks tiles of 32 cells, one thread per cell, and each lane streams its own cell's operator
 * record through the warp's ring of shared-memory stages four stencil members at a time; refused
 * likewise when it does not fit. 7168 + w / 7200 + w (mixed path, w warps per block, 1..8) select
 * the streamed schedule with two lanes per cell (each lane half of the conserved variables, 16
 * cells per warp) and a two- / three-stage ring of 4-member chunks; refused likewise. Flux only:
 * 8192 + b (b a multiple of 32 in
 * [32, 256]) selects the face-based schedule: HLLC once per face, in its owner's orientation, into
 * a face-flux array, then a per-cell gather and update (results bit-identical to the per-cell
 * schedules). At central degrees 4 to 6 and with the characteristic reconstruction the reconstruction
 * takes 1024 + b only (default 1024 + 128), and on the mixed path without the characteristic
 * reconstruction also 1536 + b (the same schedule compiled for at most 64 registers per thread, so
 * that more warps share an SM); every other reconstruction value is refused with
 * CTENO_ERR_ARG. */
int cteno_set_launch(cteno_ctx *ctx, int recon_block, int flux_block);

/* Time the candidate launch configurations (block sizes 64/128/256, on the mixed path the
 * register-capped variants at 64/128 and the staged, gather-staged and streamed reconstruction
 * schedules that fit, and the lane schedules at 128/256 threads) on the current state and keep the
 * fastest; the state is restored afterwards. The current state must be a valid one (set it first:
 * the kernels run on it). best_out[2] (may be NULL) receives the chosen values, in the convention
 * of cteno_set_launch. */
int cteno_autotune(cteno_ctx *ctx, int32_t *best_out);

/* Kernel statistics for roofline accounting: out[0] = algorithmic DRAM bytes of one
 * reconstruction launch, out[1] = of one flux/update launch, out[2] = FLOPs of one
 * reconstruction launch, out[3] = of one flux/update launch (all cells of all meshes). */
int cteno_kernel_stats(cteno_ctx *ctx, double *out);

/* Time each kernel of one step with CUDA events on the context stream (FLOP/byte accounting):
 * ms_out[0] = reconstruction (3 launches), ms_out[1] = flux/update (3 launches) of one step,
 * averaged over nsteps steps of cteno_run's graph-free path. Advances the state. */
int cteno_profile_step(cteno_ctx *ctx, int nsteps, double *ms_out);

/* Enable (1) or disable (0, default) timing of the kernels inside cteno_run's step graph: event
 * record nodes around every launch, read back by cteno_last_kernel_ms. Rebuilds the graph. */
int cteno_set_timing(cteno_ctx *ctx, int enable);

/* Device time of the last step replayed by cteno_run (timing enabled): ms_out[0] = the three
 * reconstruction launches, ms_out[1] = the three flux/update launches. Synchronises. */
int cteno_last_kernel_ms(cteno_ctx *ctx, double *ms_out);

/* Measure the FP64 and FP32 FMA throughput of the current device (TFLOP/s, 2 FLOP per FMA) with
 * independent FMA chains on every SM; about 0.5 s. Used as the ALU roofline denominator. */
int cteno_measure_alu_peak(double *fp64_tflops, double *fp32_tflops);

/* Test hook of the failure path of the bounded waits (no counterpart in the paper). With
 * limit_ns > 0 every launch of a staged reconstruction schedule (launch values 2048 + b, 3072 + b,
 * 4096, 4097) first waits, for at most limit_ns nanoseconds, on a shared-memory barrier that nothing
 * completes. The wait runs out: the kernel records the timeout in the context's error word, waits
 * (bounded) for the bulk copies it has issued, and returns; the next synchronising call returns
 * CTENO_ERR_DEVICE, as for a bulk copy that never completes. 0 (the default) turns it off; limit_ns
 * is at most 1e9. The error word of the context stays set: use a new context afterwards. */
int cteno_test_wait_timeout(cteno_ctx *ctx, int64_t limit_ns);

/* Message of the last error on this context ("" if none; "null context" for NULL). The string is
 * owned by the context and valid until its next failing call or cteno_destroy. */
const char *cteno_last_error(cteno_ctx *ctx);

/* Wait for the context's work on its stream, then free everything it allocated (device arrays,
 * staging buffers, the step graph, its events and capture stream). The borrowed stream is not
 * destroyed. NULL is a no-op. */
void cteno_destroy(cteno_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* CTENO_H */

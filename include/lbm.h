/*
 * lbm.h -- C ABI of the GB300 sparse D3Q19 TRT lattice Boltzmann library.
 *
 * The library implements the hot path of a list-based lattice Boltzmann flow
 * solver (Wittmann, Zeiser, Hager, Wellein, "Domain decomposition and
 * locality optimization for large-scale lattice Boltzmann simulations"):
 *
 *   - assembly of the sparse representation of a voxelised domain: only
 *     fluid cells are stored, in a 1-D array ordered by a numbering scheme,
 *     with an adjacency list in which bounce back is implicit (Sec. 2,
 *     "sparse representation"; Sec. 3, "Numbering scheme" and the contiguous
 *     index I_c in [1, N_f]);
 *   - the D3Q19 two-relaxation-time (TRT) stream-collide sweep over that
 *     list, pull scheme, structure-of-arrays PDFs (Sec. 1; Sec. 7, first
 *     paragraph), with FP64 mass and flux reductions.
 *
 * Conventions (the paper names D3Q19 and TRT but prints neither):
 *   - dims = {nx, ny, nz}; box cell (x, y, z) has linear index
 *     x + nx*(y + ny*z); flags[] uses that layout, 0 = fluid, 1 = solid.
 *   - velocities: q = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = face
 *     diagonals (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),(+1,0,+1),(-1,0,-1),
 *     (+1,0,-1),(-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1);
 *     opp(q) = q+1 for odd q, q-1 for even q > 0.  Weights 1/3, 1/18, 1/36.
 *   - sparse index n = I_c - 1 (0-based) of the paper's contiguous index.
 *   - PDFs are structure of arrays: f[q*N + n] at every entry point that
 *     takes or gives them (inside a state the rows are padded to L slots,
 *     see lbm_build_sparse).
 *   - adjacency adj[(i-1)*N + n], i = 1..18, is the flat source slot of the
 *     pull for direction i: i*N + m when the upwind cell x - c_i is the fluid
 *     cell m, else opp(i)*N + n (half-way bounce back, applied implicitly;
 *     Sec. 2).  The rest direction has no entry (it is always slot n).
 *   - TRT collision with body force F and Brinkman damping alpha (rho0 = 1):
 *       rho = sum g,  j = sum c g,  u = (j + F/2) / (1 + alpha/2),
 *       F_n = F - alpha u,
 *       e_q = w_q (rho + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u),
 *       f*_q = g_q - w+ (g+ - e+)_q - w- (g- - e-)_q + (1 - w-/2) 3 w_q c_q.F_n.
 *
 * Every function returns LBM_OK (0) or a negative status; lbm_last_error()
 * then returns a description (thread-local, valid until the next call from
 * the same thread).  No C++ exception crosses this interface.
 *
 * Device pointers are plain CUDA device addresses on the current device.
 * Handles (lbm_sparse, lbm_state) own device memory, taken from the
 * caller's allocator if one is set (lbm_set_allocator); they are released by
 * lbm_free.  A state refers to the sparse representation it was created
 * from, which must outlive every use of the state; lbm_free may release the
 * two in either order (a garbage collector may).  All work is queued on the
 * stream given to lbm_build_sparse (a cudaStream_t passed as void*, NULL =
 * legacy default stream); functions that return host values synchronise
 * that stream.  Distinct handles may be used from different host threads at
 * once; one handle (and a state together with the sparse representation it
 * was built from) must not be, since some calls fill caches inside it (the
 * public adjacency, captured CUDA graphs).
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LBM_OK 0
#define LBM_EINVAL (-1)      /* bad argument (null pointer, size, range) */
#define LBM_EOVERFLOW (-2)   /* index space beyond int32: box >= 2^31 cells
                                or 19*N >= 2^31 PDF slots */
#define LBM_ECUDA (-3)       /* a CUDA runtime call failed */
#define LBM_ENONFINITE (-4)  /* a reduction produced NaN or Inf */
#define LBM_ETIMEOUT (-5)    /* queued work did not finish in the time limit */
#define LBM_ENOMEM (-6)      /* device or pinned host allocation failed */
#define LBM_EFLAGS (-7)      /* a flag byte other than 0 or 1 */

/* ---- numbering schemes (Sec. 3, "Numbering scheme"; Sec. 7) ------------- */
#define LBM_ORDER_LEX 0      /* lexicographic, x fastest */
#define LBM_ORDER_BLOCKED 1  /* lexicographic with blocking: blocks of
                                block[0] x block[1] x block[2] cells visited
                                lexicographically, cells inside a block
                                lexicographically, edge blocks clipped;
                                block {1,1,1} equals LBM_ORDER_LEX */
#define LBM_ORDER_MORTON1 2  /* Z curve, 1-bit interleave: key bit 3k = x_k,
                                3k+1 = y_k, 3k+2 = z_k */
#define LBM_ORDER_MORTON2 3  /* Z curve, 2-bit groups: key bits 6k..6k+1 =
                                x bits 2k..2k+1, then y, then z */
#define LBM_ORDER_HILBERT 4  /* Hilbert curve over the enclosing 2^b cube
                                (Skilling's transform); cells outside the
                                box are skipped */

typedef struct lbm_ordering {
  int32_t kind;      /* LBM_ORDER_* */
  int32_t block[3];  /* blocking factors for LBM_ORDER_BLOCKED, each >= 1 */
  uint32_t periodic; /* bit 0: x periodic, bit 1: y, bit 2: z; a closed
                        face bounces PDFs back like a solid cell */
} lbm_ordering;

/* ---- storage precisions -------------------------------------------------- */
#define LBM_F64 0   /* f in FP64, FP64 arithmetic (the paper's form, Sec. 7) */
#define LBM_F32 1   /* f in FP32, FP32 arithmetic */
#define LBM_F32S 2  /* f - w_q in FP32, FP32 arithmetic */
#define LBM_F16S 3  /* (f - w_q) * 2^k in FP16, FP32 arithmetic */
#define LBM_BF16S 4 /* (f - w_q) * 2^k in BF16, FP32 arithmetic */
#define LBM_F64X 5  /* f in FP64; the sweep computes f - w_q exactly in 64-bit
                       fixed point (unit 2^-58) instead of FP64 instructions,
                       damping included, conserves mass exactly and agrees
                       with LBM_F64 to FP64 round-off; its adjoint steps in
                       fixed point and reverses in double-single arithmetic
                       (~48 bits); other operations run as LBM_F64 */

typedef struct lbm_sparse lbm_sparse;
typedef struct lbm_state lbm_state;

/*
 * Numbering-scheme key I(x,y,z) of every box cell (Sec. 3, "Numbering
 * scheme": a unique, not necessarily contiguous index of all cells).
 * keys_dev: device uint64[nx*ny*nz] in box layout, written on `stream`.
 * Returns LBM_EINVAL for bad dims or ordering.
 */
int lbm_ordering_keys(const int32_t dims[3], lbm_ordering ord, uint64_t* keys_dev,
                      void* stream);

/*
 * Build the sparse representation of a voxelised domain (Sec. 2-3).
 * flags:     uint8[nx*ny*nz], box layout, 0 fluid / 1 solid, read only,
 *            owned by the caller, must stay valid until this call returns;
 *            device memory, or host memory (pinned or pageable), which is
 *            first copied on `stream` into a device buffer that the call
 *            allocates and releases.
 * dims:      host int32[3], each >= 1, nx*ny*nz < 2^31 (the paper's solver
 *            has the same bound on the bounding box, Sec. 7 end).
 * ord:       numbering scheme and periodic axes.
 * stream:    cudaStream_t used by this handle and every state built on it.
 * out:       receives a library-owned handle holding, in device memory,
 *            cells[N] (box index of the fluid cell with I_c = n + 1, i.e.
 *            fluid cells ranked by key), inv[nx*ny*nz] (n, or -1 for solid)
 *            and the adjacency.  The states keep their arrays in rows of
 *            L slots, L = N rounded up to 64, so that every row starts on a
 *            128-byte boundary; the adjacency is stored in that layout
 *            (18 rows of L, entries r*L + m; 72 bytes per L), which the
 *            steps read.  When L = N that is adj[18*N] of the layout above;
 *            otherwise adj[18*N] is derived from it on its first request
 *            (lbm_sparse_info, lbm_adjoint_create, lbm_state_create_batched)
 *            and then kept.
 * The call synchronises `stream` (to learn N, and again before returning,
 * so the flags may be released afterwards).  Errors: LBM_EINVAL,
 * LBM_EFLAGS, LBM_EOVERFLOW (19*L >= 2^31), LBM_ENOMEM, LBM_ECUDA.
 */
int lbm_build_sparse(const uint8_t* flags, const int32_t dims[3], lbm_ordering ord,
                     void* stream, lbm_sparse** out);

/*
 * Read-only views of a sparse representation.  Any out pointer may be NULL.
 * The device pointers stay owned by the handle.  adj_dev is adj[18*N] of the
 * layout above; when N is not a multiple of 64 the first request builds it
 * (72 bytes per cell of device memory, one kernel on the handle's stream,
 * which the call then synchronises) and may fail with LBM_ENOMEM.
 */
int lbm_sparse_info(const lbm_sparse* sp, int64_t* n_fluid, const int32_t** cells_dev,
                    const int32_t** adj_dev, const int32_t** inv_dev);

/*
 * Create a solver state on a sparse representation: two PDF buffers (A/B,
 * pull scheme with swapped grids, Sec. 7) initialised to rest,
 * f_q = w_q (rho0 = 1).  Each buffer holds 19 rows of L slots (L = N
 * rounded up to 64, see lbm_build_sparse); the padding slots are never
 * read, and every entry point that takes or gives PDFs uses the [19][N]
 * layout above.
 * precision: LBM_F64 .. LBM_BF16S.
 * scale_exp: k of the 16-bit shifted forms, stored value (f - w_q) * 2^k
 *            rounded to nearest; 0 <= k <= 40; ignored by the other forms.
 * Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA.
 */
int lbm_state_create(const lbm_sparse* sp, int32_t precision, int32_t scale_exp,
                     lbm_state** out);

/*
 * Overwrite the current PDFs from device FP64 f_dev[19*N] (layout above),
 * converting to the state's storage form; clears the step count.
 * lbm_state_get_pdfs decodes the current PDFs into f_dev[19*N] as FP64.
 * Both are queued on the state's stream.
 */
int lbm_state_set_pdfs(lbm_state* st, const double* f_dev);
int lbm_state_get_pdfs(const lbm_state* st, double* f_dev);

/*
 * Exact copies of the current PDFs as stored, for checkpoints: raw[19*N]
 * words of the storage form (8 bytes for LBM_F64 and LBM_F64X, 4 for the
 * FP32 forms, 2 for the 16-bit forms; the shifted forms' stored
 * deviations, scaled codes for FP16/BF16), [19][N] as above, in device or
 * host memory owned by the caller.  FP64 f does not always carry a shifted
 * form's deviation: (w + d) - w differs from d where d is below ~1e-9 in
 * FP32.  lbm_state_set_raw clears the step count, as lbm_state_set_pdfs.
 * Queued on the state's stream (a pageable host buffer makes them
 * synchronous).  Not available on a batched state (LBM_EINVAL).
 */
int lbm_state_get_raw(const lbm_state* st, void* raw);
int lbm_state_set_raw(lbm_state* st, const void* raw);

/* Put the current PDFs back to rest (f_q = w_q) and clear the step count;
 * which of the two grids is current does not change. */
int lbm_state_reset(lbm_state* st);

/*
 * Per-cell Brinkman damping alpha_n >= 0 in fluid order (device FP64[N]),
 * copied into the state in its arithmetic precision (FP64 for LBM_F64 and
 * LBM_F64X, FP32 otherwise); NULL removes damping.  An LBM_F64X state also
 * keeps alpha 2^63 and e 2^63, e = (alpha/2)/(1 + alpha/2), per cell (16
 * more bytes per cell), so that its fixed-point steps and its adjoint take
 * damped cells without FP64 arithmetic; cells with alpha outside [0, 1/2)
 * take the IEEE FP64 update, with the same results to FP64 round-off.
 */
int lbm_set_damping(lbm_state* st, const double* alpha_dev);

/*
 * Advance n_steps >= 0 time steps: each is a pull through the adjacency
 * list, a TRT collision and a store to the other grid (Sec. 7: pull scheme,
 * structure of arrays, streaming stores).  omega_plus / omega_minus are the
 * even / odd relaxation rates, each in (0, 2); force is a host double[3]
 * body force, finite.  The last step of the call also writes FP64 block
 * partial sums of rho and u for lbm_reduce_flux.  Asynchronous on the
 * state's stream.  A call of more than 256 steps replays a CUDA graph of
 * 128 steps, which the state captures on a private stream the first time
 * (per grid parity and per set of rates, force and damping pointer) and
 * keeps until lbm_free; the kernels and results are those of launching
 * every step, and a stream that is itself being captured gets plain
 * launches.  The second and later steps of a call (in FP32, 16-bit and
 * fixed-point FP64-storage arithmetic) are launched with programmatic
 * dependent launch: their blocks start while the previous step ends and
 * wait in the kernel for it, which changes no result.  The first step of a
 * call waits for all earlier work on the stream as usual.  Errors:
 * LBM_EINVAL, LBM_ECUDA.
 */
int lbm_step(lbm_state* st, int32_t n_steps, double omega_plus, double omega_minus,
             const double force[3]);

/*
 * lbm_step, timed on the device: CUDA events recorded on the state's stream
 * just before and after the step launches give the device time of the
 * n_steps steps (the reducing last one included) in *ms_out, in
 * milliseconds.  Synchronises the stream (bounded by lbm_set_timeout).  The
 * events are created on the first call and kept until lbm_free.  Errors:
 * those of lbm_step, LBM_EINVAL (ms_out NULL), LBM_ETIMEOUT, LBM_ECUDA.
 */
int lbm_step_timed(lbm_state* st, int32_t n_steps, double omega_plus, double omega_minus,
                   const double force[3], double* ms_out);

/*
 * Mass and mean axial velocity of the most recent step's collision:
 * mass = sum_n rho_n and flux = (1/N) sum_n u_axis,n, returned in FP64.
 * Within each warp of 32 cells, rho - 1 and u are summed exactly as int64
 * fixed point in units of 2^-60 (2^-58 for LBM_F64X); a warp holding a
 * value of magnitude >= 1/4, NaN or Inf sums in FP64 instead.  Warp sums
 * are added in FP64 in a fixed order, so results are run-to-run identical.
 * axis in {0,1,2}.
 * Synchronises the stream (bounded by lbm_set_timeout).  Errors:
 * LBM_EINVAL (no step taken yet, bad axis), LBM_ENONFINITE, LBM_ETIMEOUT,
 * LBM_ECUDA.
 */
int lbm_reduce_flux(lbm_state* st, int32_t axis, double* mass_out, double* flux_out);

/*
 * Per-cell rho_dev[N] and u_dev[3*N] (u_dev[k*N + n]) of the most recent
 * step's collision, in FP64, recomputed from the previous grid with the
 * same arithmetic as the step.  Errors: LBM_EINVAL if no step was taken.
 */
int lbm_moments(const lbm_state* st, double* rho_dev, double* u_dev);

/* Number of steps taken since creation or the last lbm_state_set_pdfs. */
int lbm_state_steps(const lbm_state* st, int64_t* steps);

/*
 * Wait for the state's queued work, polling with a wall-clock limit of
 * timeout_s seconds (<= 0: the library default, 600 s).  Returns
 * LBM_ETIMEOUT if the work is still running at the limit; the work itself
 * is not cancelled.
 */
int lbm_synchronize(const lbm_state* st, double timeout_s);
void lbm_set_timeout(double timeout_s);

/*
 * One FP64 time step that allocates nothing.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory --
 * for example a host application that owns all of the GPU's memory and
 * hands this library only the arrays it works on, or a time-stepping loop
 * with a fixed memory budget that cannot take the device-wide
 * synchronisation and latency of a cudaMalloc.  It performs exactly what one
 * step of lbm_step does on an LBM_F64 state and what lbm_reduce_flux then
 * sums, on caller-owned arrays:
 *   f_src_dev: device FP64[19*N] PDFs before the step (layout above), read.
 *   f_dst_dev: device FP64[19*N] PDFs after the step, written; must not
 *              overlap f_src_dev.
 *   adj_dev:   device int32[18*N] adjacency, e.g. from lbm_sparse_info.
 *   n_fluid:   N, 0 <= N <= 16,777,216 (LBM_EINVAL beyond).
 *   alpha_dev: device FP64[N] Brinkman damping, or NULL for none.
 *   sums_dev:  device FP64[4], written: sum rho, sum u_x, sum u_y, sum u_z
 *              of this step's collision (flux = sum u_axis / N).
 *   stream:    cudaStream_t the work is queued on (asynchronous).
 * Its only scratch, the FP64 block partial sums (at most 65,536 blocks of
 * 256 cells), lives in a fixed 2 MiB static device array, part of the
 * library's compiled sweep code.  Under CUDA's lazy module loading (the
 * default) the driver loads that code on a device, and reserves the array
 * there, when it is first used on that device -- at the latest by this
 * entry point's first call there -- not when the library is loaded; from
 * then on the device holds the array until the process exits.  The first
 * call on a device also looks up the array's device address
 * (cudaGetSymbolAddress) with the device current.  So make the first call
 * on each device before the caller takes all of that device's memory, and
 * before any stream capture; later calls need neither.
 * Every call shares the array and it keeps the last call's contents; each
 * call overwrites the entries it reads, so nothing needs clearing, but two
 * calls that overlap on the same GPU (for example on two streams) race on
 * it.  Calls no cudaMalloc, cudaFree or other allocating routine.
 */
int lbm_step_f64_noalloc(const double* f_src_dev, double* f_dst_dev, const int32_t* adj_dev,
                         int64_t n_fluid, double omega_plus, double omega_minus,
                         const double force[3], const double* alpha_dev, double* sums_dev,
                         void* stream);

/* ---- batches of independent beds ----------------------------------------
 * Many packed beds of uneven size stepped by one launch per time step:
 * their cell lists are concatenated (each bed padded to a multiple of 2048
 * cells), each bed has its own body force, and each bed's flux is reduced
 * separately.  A bed's PDFs and flux are bit-identical to stepping it alone.
 *
 * lbm_state_create_batched: beds[n_beds] built on the same stream (they
 *   may be released afterwards; the state keeps a remapped copy of their
 *   adjacency, read from each bed's public adj[18*N], which this call builds
 *   where it is not yet built, see lbm_sparse_info).  PDF arrays of the state (lbm_state_get/set_pdfs) have the
 *   padded length N_pad; see lbm_batch_layout.  Damping, moments and the
 *   adjoint are not available on a batched state.
 * lbm_step on a batched state takes force = host double[n_beds][3];
 *   lbm_reduce_flux writes mass_out[n_beds] and flux_out[n_beds].  The
 *   launches of one lbm_step call are captured once into a CUDA graph and
 *   replayed while K, the relaxation rates, the launch shape and the L2
 *   groups (lbm_batch_groups) stay the same (forces may change between
 *   calls).
 */
int lbm_state_create_batched(const lbm_sparse* const* beds, int32_t n_beds, int32_t precision,
                             int32_t scale_exp, lbm_state** out);

/* begin_out[n_beds]: first padded index of each bed; count_out[n_beds]:
 * its fluid cells; *n_padded: N_pad.  Any out pointer may be NULL. */
int lbm_batch_layout(const lbm_state* st, int32_t* n_beds, int64_t* begin_out,
                     int64_t* count_out, int64_t* n_padded);

/* Launch shape of the non-reducing steps: block in {128, 256, 512}, cells
 * per thread in {1, 2, 4}; use_graph 0/1.  Results do not depend on it. */
int lbm_batch_config(lbm_state* st, int32_t block, int32_t cells_per_thread, int32_t use_graph);

/* L2 groups.  The beds, in layout order, are split into groups whose working
 * set (both PDF grids and the adjacency of their padded cells) fits `bytes`;
 * a bed larger than that forms a group of its own.  An lbm_step call then
 * runs all its steps on the first group, then on the next, so that each
 * group streams from L2 instead of HBM.  With one group every launch steps
 * all beds.  Either way a call of K steps is captured into a CUDA graph
 * (use_graph) when groups x K <= 2^18 launches, and otherwise launched
 * directly.  bytes = 0: one group; bytes < 0: the
 * default, 0.6 of the device's L2 (set at creation).  *n_groups_out (may be
 * NULL) receives the number of groups.  Results do not depend on it: beds
 * are independent, and each bed takes the same steps in the same order. */
int lbm_batch_groups(lbm_state* st, int64_t bytes, int32_t* n_groups_out);

/* Resident steps (mode 1).  The non-reducing steps of each L2 group that
 * holds at most C cells run as ONE cooperative launch: one 1024-thread block
 * per SM, each block reading the links of its run of the group's cells once
 * into shared memory and keeping them for all the call's steps, with a grid
 * barrier between steps.  A step then reads only PDFs from L2, not links.
 * C (*cells_out) is the SM count times the longest run (a multiple of 64
 * cells) whose links fit one block's shared memory (3,200 cells on GB300:
 * 486,400).  Switching the mode
 * re-splits the groups: with resident steps a group's working set is its two
 * PDF grids (the byte budget of lbm_batch_groups applies to those) and a
 * group holds at most C cells.  Groups larger than C, and calls of one step,
 * use the per-step launches of lbm_batch_config.  Resident calls are
 * launched directly (no graph).  Results are bit-identical to the per-step
 * launches.  mode 0: back to per-step launches.  Only for FP32 and 16-bit
 * arithmetic (LBM_F32, LBM_F32S, LBM_F16S, LBM_BF16S): LBM_EINVAL otherwise.
 * Each barrier wait gives up after 2 s, which co-residency should never
 * let happen; the next lbm_step or lbm_reduce_flux on the state then
 * returns LBM_ETIMEOUT and the PDFs are not valid.  mode -1 is a check of
 * that limit: every wait expects one block more than the grid holds and
 * gives up after 20 ms, so a call of three or more steps (two or more in
 * the cooperative launch, hence a barrier) ends with
 * LBM_ETIMEOUT reported as above.  *n_groups_out, *cells_out may be NULL. */
int lbm_batch_resident(lbm_state* st, int32_t mode, int32_t* n_groups_out, int64_t* cells_out);

/* Autotuner: times steps_per_candidate steps under each of the nine launch
 * shapes (advancing the state by 9 * (steps_per_candidate + 1) steps, whose
 * result does not depend on the shapes), keeps the fastest, and returns it
 * (ms_out[9], if given, receives each candidate's time in ms, block-major).
 * The shapes are those of the per-step launches: with resident steps on,
 * they apply only to groups above the resident capacity, so tune with
 * resident steps off. */
int lbm_batch_tune(lbm_state* st, int32_t steps_per_candidate, double omega_plus,
                   double omega_minus, const double* forces, int32_t* block_out,
                   int32_t* cpt_out, float* ms_out);

/* ---- halo exchange of a chunked list ------------------------------------
 * The flow solver cuts the fluid-cell list into equal chunks, one per rank,
 * and before every step each rank receives the PDFs of its remote links
 * into ghost cells that follow its own PDFs (Sec. 2; Fig. 1c).  This is the
 * pack side of that exchange: dst_dev[i] = src_dev[slots_dev[i]] for
 * i < count, elements of elem_bytes in {2, 4, 8}; slots_dev is a device
 * int64 array.  On one device dst_dev may point into the receiving chunk's
 * ghost run directly.  Asynchronous on `stream`.
 */
int lbm_halo_gather(const void* src_dev, const int64_t* slots_dev, int64_t count, void* dst_dev,
                    int32_t elem_bytes, void* stream);

/* ---- adjoint (reverse mode) ---------------------------------------------
 * Gradients of J = (1/N) sum_n u_axis,n, the mean axial velocity of the
 * collision of step K, with respect to the body force F and the per-cell
 * Brinkman damping alpha_n, for K steps started from a state's current
 * PDFs: lam_g_K = dJ/dg_K; lam_f_{t-1} = S^T lam_g_t (transposed pull);
 * lam_g_t = C'(g_t)^T lam_f_t (transposed TRT Jacobian).  The forward
 * states are kept as checkpoints every `stride` steps in the state's
 * storage form and recomputed between checkpoints (memory ~ (K/stride +
 * stride) states).  Adjoint arithmetic runs in the state's arithmetic
 * precision: FP64 for LBM_F64; for LBM_F64X fixed-point forward steps and
 * double-single reverse steps (lambda as pairs of FP32 values, ~48
 * significant bits, results within 1e-10 of FP64); FP32 otherwise.  Sums in
 * FP64.
 */
typedef struct lbm_adjoint lbm_adjoint;

/* Buffers for K = n_steps >= 1 steps of state st (its lattice, form and
 * damping); stride = 0 picks ceil(sqrt(K)).  The adjoint's arrays are
 * [19][N] and read the lattice's public adj[18*N], which this call builds
 * if it is not yet built (see lbm_sparse_info).  The state must outlive
 * every forward and backward pass; lbm_free may release the two in either
 * order. */
int lbm_adjoint_create(const lbm_state* st, int32_t n_steps, int32_t stride, lbm_adjoint** out);

/* Forward pass from the state's current PDFs (the state is not modified):
 * stores the checkpoints and returns J (axis in {0,1,2}).  Synchronises. */
int lbm_adjoint_forward(lbm_adjoint* adj, double omega_plus, double omega_minus,
                        const double force[3], int32_t axis, double* J_out);

/* Reverse pass of the last lbm_adjoint_forward.  dJdF_out: host double[3].
 * dJdalpha_dev: device FP64[N] (fluid order), written, or NULL.
 * dJdf0_dev: device FP64[19*N], gradient with respect to the initial PDFs,
 * written, or NULL.  May be called again (it recomputes from the
 * checkpoints).  Synchronises. */
int lbm_adjoint_backward(lbm_adjoint* adj, double dJdF_out[3], double* dJdalpha_dev,
                         double* dJdf0_dev);

/* Forward and reverse pass in one call; n_steps must equal the K the
 * adjoint was created for and st its state. */
int lbm_adjoint_step(lbm_state* st, lbm_adjoint* adj, int32_t n_steps, double omega_plus,
                     double omega_minus, const double force[3], int32_t axis, double* J_out,
                     double dJdF_out[3], double* dJdalpha_dev);

/* Release a handle returned by this library (sparse, state or adjoint);
 * NULL is a no-op.  Waits for the handle's stream before freeing. */
void lbm_free(void* handle);

/* ---- device memory --------------------------------------------------------
 * Handles take their device memory from a caller-supplied allocator when
 * one is set, else from cudaMalloc (cudaMallocAsync on the handle's stream
 * for the sparse representation and its scratch).
 *   alloc(bytes, stream, ctx) returns a device pointer aligned to at least
 *     16 bytes (cudaMalloc and PyTorch's allocator give 256), or NULL: the
 *     calling function then fails with LBM_ENOMEM.  A pointer aligned to
 *     less is given back through release and the call fails the same way
 *     (the kernels use vector accesses).
 *   release(ptr, stream, ctx) gives a block back.  It may be called while
 *     work queued on `stream` still uses the block, so the allocator must not
 *     hand the block to work on another stream before that work completes
 *     (stream-ordered reuse, as in PyTorch's caching allocator).
 * `stream` is the handle's stream (a cudaStream_t).  Set both functions, or
 * neither for the library's own.  LBM_EINVAL if only one is given, or if
 * blocks of existing handles are still live: a block goes back through the
 * allocator that gave it, so free those handles first.  The setting is
 * process-wide; do not change it while another thread uses the library. */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*lbm_free_fn)(void* ptr, void* stream, void* ctx);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void* ctx);

/* Description of the last failure on this thread ("" if none). */
const char* lbm_last_error(void);

/* ABI version, currently 2 (2 added lbm_state_get_raw and
 * lbm_state_set_raw to version 1; nothing was removed or changed). */
int32_t lbm_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */

/*
 * blip.h - C ABI of libblip: periodic cubic-blip (B-spline) orbital
 * evaluation on a GB300 (sm_103a) GPU.
 *
 * What it computes (Uejima & Maezono, arXiv:1204.1121, Sec. II.B,
 * Eqs. 11.12.24.1, 11.12.24.2 and 7): for every electron position r_j and
 * every orbital l of a precomputed coefficient table a[l, s~] on a periodic
 * grid of n1 x n2 x n3 sites,
 *
 *     psi_l(r_j) = sum_{s=1}^{64} a_{l,s(r_j)} Theta_s(r_j),
 *     Theta_s(r) = phi(g_1 - m_1) phi(g_2 - m_2) phi(g_3 - m_3),
 *
 * with g = diag(n) A^{-1} r the grid coordinates of r, A the matrix whose
 * columns are the lattice vectors, site m at r = A diag(n)^{-1} m, phi the
 * centred cubic B-spline (4 sites per direction, so s runs over 4^3 = 64
 * sites per electron), and the coefficient of site m read at m mod n.  The
 * library also returns the Cartesian gradient and Laplacian of every psi_l
 * (chain rule: grad = J^T grad_g, lap = sum_ab (J J^T)_ab d_a d_b with
 * J = diag(n) A^{-1}); these enter the local energy (Sec. II.B, step 4 of
 * the Monte Carlo step).  Many electrons of many walkers are evaluated in one
 * call, which is the batching the quasi-simultaneous update of Sec. IV.A
 * (Eq. 11.12.23.1) makes possible: every trial move of a step is judged
 * against the same frozen configuration, so all N x L evaluations are
 * independent.
 *
 * Numerics: positions are wrapped into the cell and reduced to a cell index
 * and an offset in FP64 on the GPU; weights and the 64-term contraction use
 * FP32 with FP32 accumulation (the paper runs its GPU kernel in single
 * precision, Sec. III.B and V.B).  Coefficients are stored as FP32, or as
 * BF16 / FP16 with one FP32 scale per orbital.
 *
 * Conventions for every entry point:
 *  - Return value: BLIP_OK (0) or a negative BLIP_ERR_* code; nothing is
 *    thrown and no process state other than the table is changed.
 *  - "device" pointers are CUDA global-memory addresses on the table's
 *    device; "host" pointers are ordinary (pageable or pinned) memory.
 *  - A stream is passed as void* (a cudaStream_t; NULL = the legacy default
 *    stream).  Device work is asynchronous on that stream unless stated.
 *  - The library never frees memory it did not allocate.
 */
#ifndef BLIP_H
#define BLIP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define BLIP_OK                     0
#define BLIP_ERR_INVALID_ARG       -1  /* NULL pointer, bad size or enum value   */
#define BLIP_ERR_SINGULAR_LATTICE  -2  /* lattice vectors linearly dependent     */
#define BLIP_ERR_OOM               -3  /* a device or host allocation failed     */
#define BLIP_ERR_CUDA              -4  /* a CUDA call failed (see blip_last_cuda_error) */
#define BLIP_ERR_UNSUPPORTED_DTYPE -5  /* storage kind not known                 */
#define BLIP_ERR_NO_DEVICE         -6  /* no CUDA device, or not an sm_103 part  */
#define BLIP_ERR_SCRATCH_LIMIT     -7  /* batch too large for the fixed no-allocation scratch */

/* ---- device-side status bits (reported by blip_status) ---------------- */
#define BLIP_STATUS_NONFINITE_POS  0x1 /* a position was NaN/Inf: its outputs are NaN    */
#define BLIP_STATUS_FAR_POS        0x2 /* |fractional coordinate| > 2^40: precision lost */
#define BLIP_STATUS_BAD_OFFSETS    0x4 /* walker offsets not monotone or out of range    */
#define BLIP_STATUS_TIMEOUT        0x8 /* a bounded wait in a kernel gave up             */
#define BLIP_STATUS_LAYOUT         0x10 /* a kernel's shared memory lacked the alignment its
                                           operand layout needs: it wrote no outputs       */

/* ---- storage kinds ---------------------------------------------------- */
typedef enum {
    BLIP_F32 = 0,       /* real orbitals, FP32 coefficients                          */
    BLIP_BF16 = 1,      /* real orbitals, BF16 coefficients x FP32 per-orbital scale */
    BLIP_F16 = 2,       /* real orbitals, FP16 coefficients x FP32 per-orbital scale */
    BLIP_C64 = 3,       /* complex orbitals, FP32 real/imaginary parts               */
    BLIP_BF16PAIR = 4   /* complex orbitals, BF16 real/imaginary parts x FP32 scale  */
} blip_dtype;

/* ---- normalisation of the 1-D factor phi ------------------------------ */
typedef enum {
    BLIP_NORM_BSPLINE = 0,     /* phi = cubic B-spline, phi(0) = 2/3, sum over sites = 1 */
    BLIP_NORM_ALFE_GILLAN = 1  /* phi = 3/2 x cubic B-spline, phi(0) = 1                  */
} blip_norm;

typedef struct blip_table_s *blip_table;
typedef struct blip_graph_s *blip_graph;

/*
 * blip_create - build a device-resident coefficient table.
 *
 * Defines the table a~_{l,s~} of Eq. 7 (precomputed, read once at start-up,
 * Sec. II.B) on the current CUDA device.
 *   grid[3]           n1, n2, n3 >= 4: sites along lattice vectors a_1, a_2, a_3
 *   lattice[9]        row i = lattice vector a_i in bohr (lattice[3*i + c])
 *   n_orb             orbitals (complex orbitals for BLIP_C64 / BLIP_BF16PAIR), >= 1
 *   storage           a blip_dtype
 *   norm              a blip_norm
 *   coeffs            layout [n1][n2][n3][n_orb], orbital index fastest; complex
 *                     kinds interleave (re, im) per orbital.  Element type is
 *                     double if coeffs_is_double, else float.
 *   coeffs_on_device  0: coeffs is a host pointer; 1: a device pointer
 *   out               receives the handle
 * Ownership: the library copies (and converts / quantises) the coefficients
 * into memory it owns; the caller keeps and frees its buffer.  For a device
 * source the call first waits for all work queued on the device (so a buffer
 * still being produced on any stream is complete before it is read), and it
 * synchronises the device before returning.  Errors: INVALID_ARG,
 * SINGULAR_LATTICE, UNSUPPORTED_DTYPE, OOM, CUDA, NO_DEVICE; *out is NULL on
 * error.
 */
int blip_create(const int grid[3], const double lattice[9], int n_orb, int storage, int norm,
                const void *coeffs, int coeffs_is_double, int coeffs_on_device,
                blip_table *out);

/*
 * blip_eval - values, gradients and Laplacians of all orbitals at a batch of
 * positions (Eq. 11.12.24.1 for every (j, l); Sec. IV.A batching).
 *   pos              device [n_elec][3] FP64 Cartesian positions (bohr), any
 *                    finite values (they are wrapped into the cell)
 *   n_elec           >= 0 (0 is a no-op)
 *   walker_offsets   device [n_walkers + 1] int32 prefix offsets of the walkers'
 *                    electrons in pos (offsets[0] = 0, offsets[n_walkers] =
 *                    n_elec, non-decreasing), or NULL for one walker.  Checked
 *                    on the device (BLIP_STATUS_BAD_OFFSETS).
 *   values           device [n_elec][n_orb] float (complex kinds: float2)
 *   grads            device [n_elec][3][n_orb] float (float2), or NULL
 *   laps             device [n_elec][n_orb] float (float2), or NULL
 *                    grads and laps must be both NULL (values-only mode) or
 *                    both non-NULL.
 *   stream           cudaStream_t
 * No host synchronisation and no allocation on the steady path (scratch for
 * the optional spatial sort is grown on the first call that needs it, after a
 * device synchronisation).  The sort scratch belongs to the table: sorted
 * evaluations of one table on different streams must not overlap in time.
 * Output buffers must not overlap each other or pos.  Errors: INVALID_ARG,
 * CUDA.  Device-side problems are reported through blip_status.
 */
int blip_eval(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
              int n_walkers, void *values, void *grads, void *laps, void *stream);

/*
 * blip_eval_host - blip_eval with HOST buffers, synchronous.  If every buffer
 * is page-locked (cudaHostAlloc / cudaHostRegister, e.g. torch pin_memory),
 * the kernel reads the positions and writes the outputs through the host
 * link directly, overlapping the transfers with the table gather; otherwise
 * pos (and offsets) are copied to table-owned staging buffers (grown as
 * needed), evaluated, and the outputs copied back.  Same layouts and errors
 * as blip_eval; grads/laps may be NULL together.
 */
int blip_eval_host(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
                   int n_walkers, void *values, void *grads, void *laps);

/*
 * blip_status - synchronise the table's last stream and return (and clear)
 * the OR of the device status bits raised since the last call.
 */
int blip_status(blip_table t, int *device_status);

/*
 * blip_probe_gather - a measurement aid, not an evaluation: the memory
 * traffic of one evaluation launch without its arithmetic.  For every
 * (electron, 512-byte chunk of components) item it runs the item walk, the
 * FP64 position wrap and the 64 stencil-row loads of the persistent
 * register kernel (variant 11, 8 warps per block, input order), leaves out
 * the weights and the contraction (Eq. 11.12.24.1), folds the loaded words
 * into one word per lane, and, if store_outputs != 0, writes that word to
 * the item's five output slices with the same streaming stores.  Timed next
 * to blip_eval on the same positions it gives the time the access pattern
 * itself takes (scattered 4-row columns in HBM, L2 reuse, output stores):
 * the ceiling for any kernel that reads the table in this order.  The
 * compiler is free to give the probe fewer registers (and so more resident
 * warps) than the kernel it mirrors.
 *   pos      device [n_elec][3] FP64
 *   values, grads, laps  device, laid out as for blip_eval; written only
 *            when store_outputs != 0, with meaningless contents
 * FP32 tables only; k-points are ignored.  Errors: INVALID_ARG,
 * UNSUPPORTED_DTYPE (16-bit storage), CUDA.
 */
int blip_probe_gather(blip_table t, const double *pos, int n_elec, void *values, void *grads,
                      void *laps, int store_outputs, void *stream);

/* blip_destroy - free the table and everything it owns (NULL is accepted). */
int blip_destroy(blip_table t);

/* blip_strerror - static description of an error code. */
const char *blip_strerror(int code);

/* blip_last_cuda_error - the cudaError_t behind the last BLIP_ERR_CUDA. */
int blip_last_cuda_error(void);

/*
 * blip_info - table facts for callers and benchmarks.
 *   out[0] rows stored (n1 * n2 * (n3 + 3): three ghost planes along a_3)
 *   out[1] stored row length in elements (orbital count padded)
 *   out[2] real orbital components per row (n_orb, or 2 n_orb if complex)
 *   out[3] bytes per stored element
 *   out[4] table bytes on the device
 *   out[5] storage kind, out[6] SM count, out[7] kernel variant in use
 */
int blip_info(blip_table t, long long out[8]);

/*
 * blip_set_kernel - choose the evaluation kernel and its tile shape.
 *   variant    0: automatic (tuned choice);
 *              1: register gather (each lane loads its orbitals' coefficients
 *                 straight into registers, 16 rows per batch);
 *              2: bulk-copy staging (a producer warp streams the 4 contiguous
 *                 z-rows of each stencil column into shared memory with
 *                 cp.async.bulk; consumer warps contract them);
 *              3: register gather, double-buffered batches (fully unrolled);
 *              4: register gather, double-buffered batches (rolled loop);
 *              5: cell-grouped register gather (electrons of one grid cell
 *                 share every row load; always sorts);
 *              6: as 3, with the warps of a block taking consecutive
 *                 electrons of one chunk group and the row loads cached in
 *                 L1 (shares rows between neighbours of a sorted batch);
 *              7: as 6, the warps of a block stepping through the row
 *                 batches in lockstep (one block barrier per batch);
 *              8: staged tiles for dense batches (always sorts): the union
 *                 of the stencil rows of 2 x 2 x chunks grid cells is copied
 *                 into shared memory once (cp.async.bulk, one 512-byte chunk
 *                 of components at a time) and every electron of those
 *                 cells is contracted from there; not with k-points;
 *              9: as 3 with two row batches in flight (FP32 tables, one
 *                 chunk per warp);
 *             10: split stencil for small, latency-bound launches: 4 warps
 *                 per (electron, chunk), one a_1 slab of 16 sites each, all
 *                 16 rows loaded at once, the partial sums added in a fixed
 *                 order (agrees with the other variants to rounding, not
 *                 bitwise); not with k-points;
 *             11: as 9 with a grid of resident warps that walk the (electron,
 *                 chunk) items; each warp prefetches the next electron's
 *                 position (cp.async) and runs its FP64 wrap while the
 *                 current rows are in flight (FP32 tables, one chunk per
 *                 warp; not with k-points);
 *             12: tensor cores for dense batches (always sorts): parts of up
 *                 to 25 electrons from at most 5 consecutive cells along a_3
 *                 of one grid column share the union of their stencils,
 *                 16 columns x 8 rows; the contraction over it is a matrix
 *                 product on the tensor cores (tcgen05, accumulators in
 *                 tensor memory), the coefficients as stored (16-bit tables)
 *                 or, for FP32 tables, as two FP16 planes of a / s_l with
 *                 s_l a power of two (22 significant bits, made on first
 *                 use), times the weights split into two 16-bit parts;
 *                 agrees with the other variants to rounding, not bitwise;
 *                 not with k-points
 *   chunks     variants 1, 3, 4, 6, 7: orbital chunks (32 lanes x 16 bytes) per
 *              warp, 1..3 (1 for 16-bit storage); variants 9, 11: 1; variant 2: consumer warps
 *              per CTA, 1..8; variant 5: electrons per group, 2 or 4;
 *              variant 8: tile cells along a_3, 2 or 4; variants 10, 12: 1
 *   warps      variants 1, 3, 4, 6, 7, 9, 11: warps per block, 1..16; variant 2:
 *              shared-memory pipeline stages, 2..32; variant 5: warps per
 *              block, 1..8; variant 8: consumer warps per CTA, 12 or 16;
 *              variant 10: 4; variant 12: 1
 *   sort       0: electrons in input order; 1: sort by grid cell first (L2
 *              reuse for large batches); 2 (variants 1, 3, 4, 9, 11): sorted, and
 *              the warps' work ordered by orbital chunk group first, so the
 *              warps in flight cover more electrons with a smaller slice of
 *              each row
 * Errors: INVALID_ARG for values outside those sets; variant 12 may also
 * return OOM or CUDA (its column list and, for FP32 tables, its two FP16
 * planes are made here).
 */
int blip_set_kernel(blip_table t, int variant, int chunks, int warps, int sort);

/*
 * blip_autotune - time each kernel configuration on this batch shape and keep
 * the fastest for batches of this size class (the bit length of n_elec) and
 * output mode (values only, or all five outputs).  Every candidate is timed
 * once (median of 3 for launches under 0.2 ms); the 16 fastest, median of 7
 * runs; those within 5 % of the best
 * median, 15 more runs each, interleaved; of these the earliest in the
 * candidate list whose median is within 1 % of the best is kept (a stable
 * choice when the gap is below the timing noise).  Each run follows a read
 * sweep of a 256 MB scratch that leaves only its clean lines in L2 (the
 * scratch is allocated for the call).  Same arguments as blip_eval (the
 * outputs are overwritten).  Synchronises the stream; must not be called
 * during stream capture.  *chosen receives {variant, chunks, warps, sort}.
 */
int blip_autotune(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
                  int n_walkers, void *values, void *grads, void *laps, void *stream,
                  int chosen[4]);

/*
 * blip_set_kpoints - Bloch orbitals for a complex table.
 *
 * With k-points set, complex orbital l in [koffs[q], koffs[q + 1]) is
 * psi_l(r) = exp(i k_q . r) u_l(r), where u_l is the periodic blip expansion
 * held in the table (Eqs. 11.12.24.1 and 11.12.24.2) and
 * k_q = 2 pi A^{-T} kappa_q.  blip_eval then returns psi, grad psi =
 * e^{ik.r}(grad u + i k u) and lap psi = e^{ik.r}(lap u + 2 i k.grad u -
 * |k|^2 u).  This lets a primitive-cell table with n_k k-points stand in for
 * a supercell table n_k times larger (the paper's TiO2 orbitals are complex,
 * Sec. VI.A; the phase convention is not stated there).
 *   n_k      0 (clear) .. 64
 *   kfrac    host [n_k][3] kappa_q in reciprocal-lattice units
 *   koffs    host [n_k + 1] complex-orbital offsets, 0 = koffs[0] <= ... <=
 *            koffs[n_k] = n_orb
 * The phase uses the unwrapped fractional coordinates, reduced mod 1 in
 * FP64.  Errors: INVALID_ARG, UNSUPPORTED_DTYPE (real tables).  The bulk-copy,
 * staged-tile, split-stencil, persistent and tensor-core kernels (variants
 * 2, 8, 10, 11 and 12) have no Bloch epilogue and are not used while
 * k-points are set.
 */
int blip_set_kpoints(blip_table t, int n_k, const double *kfrac, const int *koffs);

/*
 * blip_eval_ratio - fused quasi-simultaneous ratio (real orbitals).
 *
 * For the trial move r'_j of each electron (Sec. IV.A, Eq. 11.12.23.1) the
 * determinant ratio is the new orbital row dotted with column j of the
 * inverse Slater matrix, xi_j = sum_l psi_l(r'_j) (D^{-1})_{lj} (the
 * identity behind the Sherman-Morrison update, Sec. VI.D); the drift and
 * kinetic terms need the same contraction of the gradient and Laplacian.
 * This call evaluates the orbitals (Eq. 11.12.24.1) and contracts them on the
 * chip, writing five numbers per electron instead of 5 n_orb:
 *   inv_cols   device [n_elec][n_orb] float: for electron j, the column
 *              (D^{-1})_{. j} of its own walker's and spin's inverse
 *   ratio      device [n_elec][5] float: sum_l {psi, d/dx psi, d/dy psi,
 *              d/dz psi, lap psi}_l(r'_j) inv_cols[j][l]
 *   values     device [n_elec][n_orb] float for the new rows psi_l(r'_j)
 *              (needed to update D^{-1} after an accepted move), or NULL
 *   sort       0: input order; 1: grid-cell order, and for dense batches
 *              (n_elec >= half the grid cells) the tensor cores: without
 *              `values`, the orbital sum first (sum_k W_o[k] sum_l a[k][l]
 *              inv_cols[j][l] over the union rows k of up to 25 electrons,
 *              the columns split into two 16-bit parts; for FP32 and FP16
 *              tables scaled per electron by a power of two from a pre-pass
 *              over the columns); with `values`, the evaluation kernel's
 *              products contracted in its epilogue.  Both accumulate in FP32
 *              and round differently from the CUDA cores, within the
 *              per-output bound 1.6e-5 sum_s |W_o(s)| |a_ls| carried through
 *              the column (plus the column's 16-bit split);
 *              2: grid-cell order on the CUDA cores only
 * The tensor-core path builds its operand planes and tensor maps on first
 * use, and the per-electron scales of FP32 / FP16 tables need n_elec floats
 * of scratch, allocated when a larger batch first arrives: make the first
 * call of a batch size outside stream capture (under capture without them
 * the call falls back to the CUDA cores or to the epilogue contraction).
 * Other arguments as blip_eval.  Deterministic (fixed reduction order).
 * Errors: INVALID_ARG, UNSUPPORTED_DTYPE (complex tables), OOM, CUDA.
 */
int blip_eval_ratio(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
                    int n_walkers, const float *inv_cols, float *ratio, float *values, int sort,
                    void *stream);

/*
 * blip_sm_update - Sherman-Morrison update of the inverse Slater matrices of
 * a batch of walkers after one accepted move each (Sec. VI.D).
 *
 * Row j of walker w's matrix D_w (D[j][l] = psi_l(r_j)) is replaced by the
 * new orbital row psi' (e.g. the `values` output of blip_eval_ratio).  With
 * w_k = sum_l psi'_l Dinv[l][k] (w_j = xi, the acceptance ratio):
 *     Dinv'[l][k] = Dinv[l][k] - Dinv[l][j] (w_k - delta_jk) / w_j.
 *   n_walkers  >= 0 (<= 65535)
 *   n          matrix order (electrons of one spin = orbitals), 1..32768
 *   dinv       device [n_walkers][n][n] float, Dinv[l][k] row-major, updated
 *              in place
 *   rows       device [n_walkers][n] float: the new row of each walker
 *   cols       device [n_walkers] int32: j, or -1 to leave the walker as is
 *   work       device [n_walkers][2 n] float scratch, caller-owned
 *   stream     cudaStream_t
 * The move must have xi != 0 (a rejected or impossible move is not applied
 * by the caller).  FP32 arithmetic; repeated updates accumulate rounding, so
 * QMC codes recompute the inverse from scratch periodically.  Errors:
 * INVALID_ARG, CUDA.
 */
int blip_sm_update(int n_walkers, int n, float *dinv, const float *rows, const int *cols,
                   float *work, void *stream);

/*
 * blip_test_stall_pipeline - test hook for the failure path (no counterpart
 * in the paper).  With on != 0, launches of the bulk-copy, staged-tile and
 * tensor-core kernels (variants 2, 8 and 12) on this table stall their own
 * pipeline: the consumers (the tensor-core kernel's MMA thread) never release
 * the first stage, so the producer's bounded wait runs out, it drains the
 * copies it has in flight, and the other roles' bounded waits run out too.
 * The launch returns after a few seconds with BLIP_STATUS_TIMEOUT set and
 * undefined outputs; the context stays usable.  on = 0 restores normal
 * operation.  Nothing faults, traps or spins without a bound.
 */
int blip_test_stall_pipeline(blip_table t, int on);

/*
 * blip_set_l2_residency - keep (a share of) the table resident in L2 across
 * evaluations.  For tables that fit in the persisting part of L2 - a
 * primitive-cell table with k-points (blip_set_kpoints) instead of a
 * supercell table, Sec. VI.C's cache trials - the coefficient rows of every
 * launch are then L2 hits even though the outputs stream through L2.
 *   fraction   0: off; (0, 1]: the share of the table's bytes in the window
 * The window is capped by the device's largest access-policy window, the
 * persisting part by its persisting-L2 maximum (a window larger than that is
 * marked persisting in proportion, the hit ratio).  This sets the context's
 * persisting-L2 limit (cudaLimitPersistingL2CacheSize), a per-context setting
 * that ends with the context; turning the window off or destroying the table
 * resets it to 0 and returns the persisting lines to normal.  Evaluation
 * launches on a stream created by the caller carry the window (the stream's
 * own window is restored after each launch); launches on the legacy default
 * stream (NULL) run without it.  Outputs are unchanged.  Errors:
 * INVALID_ARG (fraction outside [0, 1], another device current, no
 * persisting L2 on the device), CUDA.
 */
int blip_set_l2_residency(blip_table t, double fraction);

/*
 * blip_probe_l2_read - a measurement aid, not an evaluation: read the device
 * buffer buf (bytes, a multiple of 16, 16-byte aligned) reps times in one
 * launch, every load through L2 with L1 bypassed.  Timed on a buffer that
 * fits in L2 it gives the L2 -> SM read bandwidth that bounds evaluations of
 * L2-resident tables.  Asynchronous on stream; nothing is written.  Errors:
 * INVALID_ARG, CUDA.
 */
int blip_probe_l2_read(const void *buf, size_t bytes, int reps, void *stream);

/*
 * blip_test_fail_alloc - test hook for the out-of-memory path (no
 * counterpart in the paper).  With n >= 0 the library's device allocations
 * succeed n more times and the next one fails with cudaErrorMemoryAllocation
 * without calling cudaMalloc; the entry point that asked for it returns
 * BLIP_ERR_OOM after releasing what it had allocated (blip_create leaves
 * *out NULL), and the hook disarms itself.  n < 0 disarms it.  The setting
 * is process-wide.  Nothing is allocated, faulted or left in a bad state.
 */
int blip_test_fail_alloc(int n);

/*
 * blip_graph_create - capture a fixed evaluation into a CUDA graph.
 * The graph evaluates pos[0 .. n_elec) with the given buffers in launches of
 * per_launch electrons each (per_launch = 1 reproduces one-at-a-time,
 * particle-by-particle evaluation; per_launch = n_elec one batched launch).
 * The pointers are baked into the graph and must stay valid.
 */
int blip_graph_create(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
                      int n_walkers, void *values, void *grads, void *laps, int per_launch,
                      blip_graph *out);
int blip_graph_launch(blip_graph g, void *stream);
int blip_graph_destroy(blip_graph g);

/*
 * blip_eval_sorted_noalloc - blip_eval with the electrons sorted by grid cell,
 * for callers that must not allocate device memory during an evaluation.
 *
 * No counterpart in the paper: this is a service of the library.  Some
 * callers cannot let a library call cudaMalloc: code that is being recorded
 * into a CUDA graph (an allocation is not allowed in the middle of a stream
 * capture), and Monte Carlo drivers or frameworks that hand all device memory
 * to their own pool at start-up and run with a fixed budget (there a new
 * allocation can fail, fragment the pool, or synchronise the device in the
 * middle of a step).  blip_eval with the sort enabled grows its scratch with
 * cudaMalloc the first time a batch needs more; this entry point instead
 * takes the sort's scratch (histogram, keys, permutation) from one fixed
 * 8 MiB device buffer built into the library, and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 * Arguments, layouts, results and errors are those of blip_eval; the
 * evaluation kernel is the table's current choice (blip_set_kernel /
 * blip_autotune), always run on the cell-sorted order.
 * Limit: the scratch needed is about 4 (n1' n2' n3 + 1) + 8 n_elec bytes,
 * with n1', n2' the grid sizes rounded up to multiples of 32 (the sort's
 * 32 x 32-column super-bricks); a batch that needs more than 8 MiB returns
 * BLIP_ERR_SCRATCH_LIMIT and does nothing (about 0.8 million electrons on the
 * 72 x 72 x 48 grid).
 * The table's device must be the current device.  The first call on a device
 * looks up the buffer's device address (which may load the library's code on
 * that device); make that first call before any stream capture.
 * Every device that loads the library holds the 8 MiB buffer until the
 * process exits.  All calls on a device share the one buffer and it keeps the
 * last call's contents (the call clears what must start at zero itself), so
 * calls whose work can overlap on the GPU - on different streams without an
 * ordering between them, or from several threads - race on it and give wrong
 * results; order them on one stream.
 */
int blip_eval_sorted_noalloc(blip_table t, const double *pos, int n_elec,
                             const int *walker_offsets, int n_walkers, void *values,
                             void *grads, void *laps, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BLIP_H */

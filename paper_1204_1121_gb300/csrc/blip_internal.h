// Internal declarations shared by the CUDA translation units of libblip.
// Not part of the public ABI (include/blip.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace blip {

// Element kinds of the stored table.
enum Elem { ELEM_F32 = 0, ELEM_BF16 = 1, ELEM_F16 = 2 };

// Kernel variants.
enum Variant {
    VAR_AUTO = 0,
    VAR_REGISTER = 1,         // batches of 16 rows, loads then contraction
    VAR_BULK = 2,             // bulk-copy producer/consumer pipeline
    VAR_REGISTER_PIPE = 3,    // double-buffered batches, fully unrolled
    VAR_REGISTER_ROLLED = 4,  // double-buffered batches, rolled loop
    VAR_GROUPED = 5,          // electrons of one cell share each row load (sorted)
    VAR_REGISTER_L1 = 6,      // double-buffered; a block's warps take consecutive
                              // electrons of one chunk group and share rows via L1
    VAR_REGISTER_LOCKSTEP = 7,// as 6, the block's warps in lockstep per row batch
    VAR_STAGED = 8,           // 2 x 2 x TZ cell tiles: union rows staged in shared
                              // memory, every electron of the tile contracted there
    VAR_REGISTER_PIPE3 = 9,   // as 3 with two batches in flight (FP32, 1 chunk per warp)
    VAR_SPLIT = 10,           // 4 warps per (electron, chunk), one a_1 slab of the
                              // stencil each: one round of latency (small launches)
    VAR_REGISTER_PERSIST = 11,// as 9 with resident warps that walk the items and
                              // prefetch the next electron's geometry (no k-points)
    VAR_TENSOR = 12           // parts of up to 25 electrons of <= 5 cells of one grid
                              // column: tensor-core products over their union rows
};

constexpr int kMaxKpoints = 64;   // a 4 x 4 x 4 k-point mesh

// Cell geometry, prepared once on the host in FP64.
struct Geometry {
    int n[3];          // grid points along a_1, a_2, a_3
    double ainv[9];    // A^{-1}, row-major: u_a = sum_c ainv[3a + c] r_c
    float J[9];        // J = diag(n) A^{-1}, row-major J[3a + c]
    float M[6];        // J J^T entries xx, yy, zz, xy, xz, yz
    float norm;        // 1, or (3/2)^3 for phi(0) = 1 blips
};

// Spatial sort key of grid cell (x, y, z): 8 x 8 bricks of whole a_3
// columns, grouped 4 x 4 into super-bricks of 32 x 32 columns; super-bricks
// in row-major order, bricks inside a super-brick row-major, columns inside
// a brick row-major, a_3 fastest.  A brick's neighbour along a_1 then comes 4
// bricks later in the order (not a whole row of bricks later), so most of
// the halo rows their stencils share are still in L2 when the second brick
// reads them.
__host__ __device__ inline int sort_cell_key(const Geometry &g, int x, int y, int z)
{
    const int nsy = (g.n[1] + 31) >> 5;                      // super-bricks along a_2
    const int sb = (x >> 5) * nsy + (y >> 5);
    const int br = ((x >> 3) & 3) * 4 + ((y >> 3) & 3);
    const int col = (x & 7) * 8 + (y & 7);
    return ((sb * 16 + br) * 64 + col) * g.n[2] + z;
}

// Number of cell keys (the key of positions without a cell is this number).
__host__ __device__ inline long long sort_key_count(const Geometry &g)
{
    return (long long)((g.n[0] + 31) >> 5) * ((g.n[1] + 31) >> 5) * 1024 * g.n[2];
}

// Per-electron geometry computed once by the sort pre-pass (FP64 wrap done
// there): base cell, FP32 offsets and status bits, stored in slot order.
struct __align__(16) ElecGeo {
    int i[3];
    int bad;
    float t[3];
    float pad;
};

// Everything one evaluation launch needs (passed by value as the kernel
// parameter).
struct EvalParams {
    const void *table;      // rows [n1][n2][n3 + 3][row_stride] of the stored element
    const float *scales;    // [Lreal] per-component scale, or nullptr
    long long row_stride;   // stored elements per row (padded)
    int Lreal;              // real components per row (n_orb, or 2 n_orb if complex)
    int nchunk;             // 16-byte-per-lane chunks per row: ceil(Lreal / (32 * VEC))
    int groups;             // chunk groups per electron: ceil(nchunk / chunks per warp)
    long long items;        // n_elec * groups
    int group_major;        // register kernels: items ordered chunk group slowest
    Geometry geo;
    const double *pos;      // [n_elec][3]
    int n_elec;
    const int *perm;        // evaluation order of the electrons, or nullptr
    const ElecGeo *georec;  // per-slot geometry from the sort pre-pass, or nullptr
    const int *offsets;     // [n_walkers + 1] or nullptr
    int n_walkers;
    float *values;          // [n_elec][Lreal]
    float *grads;           // [n_elec][3][Lreal] or nullptr (values only)
    float *laps;            // [n_elec][Lreal] or nullptr
    int vec_out;            // 1: outputs may be written with 16-byte stores
    int *status;            // device status word (atomicOr)
    // Bloch phase (complex tables only): complex orbitals [koff[q], koff[q+1])
    // carry exp(i k_q . r), k_q = 2 pi A^{-T} kappa_q; n_k = 0 for none.
    int n_k;
    int koff[kMaxKpoints + 1];
    double kfrac[kMaxKpoints][3];
    float kcart[kMaxKpoints][3];
};

// Stored elements per 16-byte vector.
inline int elem_vec(int elem) { return elem == ELEM_F32 ? 4 : 8; }
inline int elem_bytes(int elem) { return elem == ELEM_F32 ? 4 : 2; }

// Launch a register-gather kernel: variants VAR_REGISTER, _PIPE, _ROLLED,
// _L1, _LOCKSTEP and _PIPE3.  chunks in {1, 2, 3} (1 for 16-bit elements,
// and for _PIPE3); warps in [1, 16].
cudaError_t launch_eval(const EvalParams &p, int elem, int variant, int chunks, int warps,
                        cudaStream_t stream);

// Register-gather instantiations (blip_reg_*.cu); pipe 0-5: batch, pipelined,
// rolled, L1-shared, lockstep, two batches in flight.
cudaError_t launch_register_f32_c1(const EvalParams &p, int warps, int pipe, cudaStream_t stream);
cudaError_t launch_register_f32_c2(const EvalParams &p, int warps, int pipe, cudaStream_t stream);
cudaError_t launch_register_f32_c3(const EvalParams &p, int warps, int pipe, cudaStream_t stream);
cudaError_t launch_register_bf16(const EvalParams &p, int warps, int pipe, cudaStream_t stream);
cudaError_t launch_register_f16(const EvalParams &p, int warps, int pipe, cudaStream_t stream);

// Persistent two-batch register kernel (blip_persist.cu): FP32 tables, one
// chunk per warp, no Bloch epilogue; at most as many blocks as fit at once.
cudaError_t launch_persist(const EvalParams &p, int warps, int sm_count, cudaStream_t stream);
// The measurement probe of the same kernel (input order, FP32): geometry and
// row loads without the arithmetic; store = also write the five outputs.
cudaError_t launch_probe(const EvalParams &p, int warps, int sm_count, bool store, cudaStream_t stream);

// Launch the bulk-copy kernel: tw chunks per tile (consumer warps, 1..8),
// `stages` shared-memory stages, ctas_per_sm persistent CTAs per SM.
// stall != 0 is a test hook: the consumers never release the first stage, so
// the bounded waits run out and BLIP_STATUS_TIMEOUT is raised.
cudaError_t launch_bulk(const EvalParams &p, int elem, int tw, int stages, int ctas_per_sm,
                        int sm_count, int stall, cudaStream_t stream);
size_t bulk_smem_bytes(int tw, int stages);

// Launch the fused ratio kernel (one warp per electron): ratio[e][0..4] =
// sum_l {psi, dpsi/dx, dpsi/dy, dpsi/dz, lap psi}_l(r_e) cols[e][l]; also
// writes p.values if it is not null.  p.grads/p.laps are ignored.
cudaError_t launch_ratio(const EvalParams &p, int elem, const float *cols, float *ratio,
                         int warps, cudaStream_t stream);

// Optional spatial sort: writes perm[n_elec] (electron ids ordered by grid
// brick).  scratch must hold sort_scratch_bytes(n_elec) bytes.
size_t sort_scratch_bytes(int n_elec, const Geometry &geo);
cudaError_t launch_sort(const Geometry &geo, const double *pos, int n_elec, void *scratch,
                        int **perm_out, cudaStream_t stream, ElecGeo *rec_by_e = nullptr,
                        ElecGeo *rec_by_slot = nullptr);
// After launch_sort: the electrons' cell keys and, per key, one past its last
// slot in the sorted order.
void sort_views(const Geometry &geo, int n_elec, void *scratch, const int **keys,
                const int **cell_end);

// Launch the cell-grouped kernel (needs the sort): warps whose slot leads a
// group of up to `group` (2 or 4) electrons of the same cell evaluate them
// together, reading each stencil row once for the whole group.
cudaError_t launch_grouped(const EvalParams &p, int elem, int group, int warps, const int *keys,
                           const int *cell_end, cudaStream_t stream);

// Opaque 128-byte tensor-map (TMA descriptor) storage.
struct alignas(64) TmaDesc {
    unsigned long long w[16];
};

// Tensor map of a stored table for the staged-tile kernel with tile depth tz:
// the table as a 2-D tensor [rows][row_stride] of its element, box = one
// 512-byte chunk x (tz + 3) rows.  Returns cudaSuccess or an error.
cudaError_t make_staged_tmap(const void *table, int elem, long long row_stride, long long rows,
                             int tz, TmaDesc *out);

// Launch the staged-tile kernel (needs the sort): tiles of 2 x 2 x tz cells
// (tz = 2 or 4), the union of their stencil rows copied into shared memory
// chunk by chunk, all electrons of a tile contracted from there by cw (12 or
// 16) consumer warps.  tmap comes from make_staged_tmap for the same table
// and tz.  stall != 0 is the same test hook as for launch_bulk.
cudaError_t launch_staged(const EvalParams &p, int elem, int tz, int cw, const int *cell_end,
                          const TmaDesc &tmap, int sm_count, int stall, cudaStream_t stream);

// Tensor map of the operand planes of the tensor-core kernel: a 2-D tensor
// [rows_total][row_stride] of 16-bit elements (elem BF16 or F16), box 64
// elements x 8 rows, 128-byte swizzle.
cudaError_t make_tc_tmap(const void *base, int elem, long long row_stride, long long rows_total,
                         TmaDesc *out);
// The two FP16 planes of an FP32 table for the tensor-core kernel: scales[l]
// = the smallest power of two >= max |a_l| (1 for zero components), planes
// [2][rows][row_stride] = RN(a / s_l) and RN(a / s_l - hi).  bits: scratch of
// row_stride words.
cudaError_t launch_split_pairs(const float *src, long long rows, long long row_stride, int Lreal,
                              unsigned int *bits, float *scales, void *dst, cudaStream_t stream);
// The 5-D view of the same operand for wide boxes: components within a
// 64-component slab, rows of a grid column (n3 + 3), grid columns (n1 n2),
// slabs, planes; box 64 x 8 x 4 x box_slabs x 1 (box_slabs 2: the 8 KB boxes
// of the evaluation kernel; 1: the 4 KB boxes of the ratio kernel's K-major
// stages).
cudaError_t make_tc_tmap5(const void *base, int elem, long long row_stride, int n12, int n3,
                          int planes, long long plane_rows, int box_slabs, TmaDesc *out);
// Launch the tensor-core kernel (needs the sort): elem = ELEM_BF16 / ELEM_F16
// (tmap over the table, p.scales its per-component scales or null) or ELEM_F32
// (tmap over its two FP16 planes, each plane_rows rows, p.scales their
// power-of-two scales); tmap5: the 5-D view (or null: 1 KB boxes only);
// cols: the ncols column keys in sort order; col_ctr: one device int, the
// CTAs' column counter (set to 0 by an async memset before the kernel).
// Ratio mode when ratio is not
// null: rcols [n_elec][Lreal] the inverse columns, ratio [n_elec][5] the
// contraction, p.values the new rows or null, p.grads and p.laps null.
cudaError_t launch_tc(const EvalParams &p, int elem, const int *cell_end, const int *cols,
                      int ncols, long long plane_rows, const TmaDesc &tmap, const TmaDesc *tmap5,
                      int *col_ctr, int sm_count, int stall, cudaStream_t stream,
                      const float *rcols = nullptr, float *ratio = nullptr);

// Launch the tensor-core ratio kernel (blip_ratio_tc.cu; needs the sort, as
// launch_tc): ratio [n_elec][5] = the contraction of each electron's orbital
// outputs with its column rcols [n_elec][Lreal], the orbital sum on the
// tensor cores; p.values, p.grads and p.laps null.  tmap5k: the 5-D view with
// box_slabs 1 (or null: 1 KB boxes only).  sig: device scratch of n_elec
// floats (the columns' scales, written by a pre-pass; unused for BF16).
cudaError_t launch_ratio_tc(const EvalParams &p, int elem, const int *cell_end, const int *cols,
                            int ncols, long long plane_rows, const TmaDesc &tmap,
                            const TmaDesc *tmap5k, int *col_ctr, int sm_count, int stall,
                            cudaStream_t stream, const float *rcols, float *ratio, float *sig);

// Launch the split-stencil kernel: a block of 4 warps per (electron, chunk),
// warp q contracting the 16 sites of a_1 slab q, partial sums added in a
// fixed order (p.groups must equal p.nchunk).
cudaError_t launch_split(const EvalParams &p, int elem, cudaStream_t stream);

// Sherman-Morrison update of n_walkers inverses after one accepted move each
// (blip_sm.cu); work holds [n_walkers][2 n] floats.
cudaError_t launch_sm_update(int n_walkers, int n, float *dinv, const float *rows, const int *cols,
                             float *work, cudaStream_t stream);

// Read bytes of buf through L2 (no writes): afterwards L2 holds clean lines
// of buf only (the autotuner's cold start).
cudaError_t launch_l2_sweep(const void *buf, size_t bytes, int sm_count, cudaStream_t stream);
// Read bytes of buf reps times through L2, L1 bypassed (a measurement aid).
cudaError_t launch_l2_read(const void *buf, size_t bytes, int reps, int sm_count,
                           cudaStream_t stream);

// Table construction kernels (blip_table.cu).
// Convert rows [row0, row0 + nrows) of a source table [n1*n2*n3][Lreal]
// (src points at row row0) into the FP32 ghost-plane layout.
cudaError_t launch_stage_rows(const void *src, int src_is_double, long long row0, long long nrows,
                              const Geometry &geo, int Lreal, long long row_stride, float *dst,
                              cudaStream_t stream);
// Per-component max |a| over the stored FP32 table (ghost rows included).
cudaError_t launch_absmax(const float *table, long long rows, long long row_stride, int Lreal,
                          unsigned int *absmax_bits, cudaStream_t stream);
// scales[l] from the max |a| bits (pairs = 1: complex pairs share one scale).
cudaError_t launch_make_scales(const unsigned int *absmax_bits, int Lreal, int pairs,
                               float *scales, cudaStream_t stream);
// Quantise the FP32 table into BF16 / FP16 with the per-component scales.
cudaError_t launch_quantize(const float *src, long long rows, long long row_stride, int Lreal,
                            const float *scales, int elem, void *dst, cudaStream_t stream);

}  // namespace blip

// Staged-tile evaluation kernel for dense sorted batches.
//
// Electrons in neighbouring cells share most of their 64 stencil rows (Eq. 7:
// the 4 x 4 x 4 sites around the cell).  When a batch holds many electrons
// per grid cell (many walkers moved in one quasi-simultaneous step,
// Sec. IV.A), this kernel reads the rows of a small block of cells once into
// shared memory and contracts every electron of the block from there: the
// L2-to-SM traffic falls from 64 rows per electron to the block's union of
// rows divided by its electron count.
//
// A tile is 2 x 2 x TZ cells; the union of its stencils is 5 x 5 x (TZ + 3)
// rows (stencil columns along a_3 are contiguous thanks to the ghost
// planes).  One stage holds that union restricted to one 512-byte chunk of
// orbital components (128 FP32 or 256 16-bit components), laid out
// [column (5 x 5)][z-row (TZ + 3)][512 bytes].
//
// Persistent grid, one CTA per SM: one producer warp and 12 or 16 consumer
// warps.
//   * producer: for each tile (static round robin), each part of the tile's
//     electrons (at most 32, or 24 with TZ = 2, so their weights fit) and
//     each chunk, waits for a free stage (a ring of 2 stages, or 3 with
//     TZ = 2) and copies the union with 25 tiled tensor copies (TMA), one
//     512-byte x (TZ + 3)-row box per stencil column, the stage's mbarrier
//     counting the bytes.  (With one 512-byte bulk copy per row instead, the
//     producer needed about 115 cycles per copy and the consumers waited for
//     stages a third of the time; with one box per column the producer
//     mostly waits for free stages.)  It also asks L2 to prefetch the whole
//     union rows of its next tile, so that those copies hit in L2.
//   * consumers (CW = 12 or 16 warps): per part, form the combined weights
//     of its electrons in shared memory (electron j by warp j mod CW), then
//     per stage contract them (one warp per electron, 16 bytes of each row
//     per lane, 5 FMAs per component and site in the same site order as the
//     register kernels, so results are bitwise identical) and store the
//     outputs.  Electrons go to warps round robin, the rotation carried from
//     stage to stage, so the warps of a CTA stay level within a part and
//     drift across at most two stages (handing the electrons out from a
//     shared counter instead kept the warps in step at every stage boundary
//     and was measured about 9 % slower).  Units of two electrons - pairs of
//     one cell sharing each row load, or any two - were measured 0-24 %
//     slower: the second set of accumulators takes registers that the loads
//     in flight need.
// The electrons of a tile are four contiguous slot ranges of the sorted
// order (one per (a_1, a_2) column of the tile: the brick-major sort key
// runs along a_3 fastest); positions without a cell sit in the last bucket
// and get NaN outputs.  Every wait is bounded (about two seconds of global
// time): a wait that runs out sets BLIP_STATUS_TIMEOUT and the CTA winds
// down, the producer first draining the copies it has in flight.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "blip_mbar.cuh"

namespace blip {

namespace {

using namespace dev;
using namespace mb;

constexpr int kTX = 2, kTY = 2;                  // tile cells along a_1, a_2
constexpr int kCX = kTX + 3, kCY = kTY + 3;      // union columns along a_1, a_2
constexpr int kSlice = 512;                      // bytes of one row per stage

// Ring depth and electrons per part: the smaller TZ = 2 stages leave room
// for a third stage (a deeper pipeline) at the price of smaller parts.
template <int TZ> struct TileCfg {
    static constexpr int S = TZ == 2 ? 3 : 2;
    static constexpr int ECAP = TZ == 2 ? 24 : 32;
};

// Weights of one electron of the current part.
struct __align__(16) ElecW {
    float4 w4[64];   // value and Cartesian gradient weights per site
    float wl[64];    // Laplacian weights
    int base;        // stage row of stencil column (0, 0), z-row 0
    int e;           // output index
    int pad[2];
};

struct StagedArgs {
    const int *cell_end;   // sort: one past the last slot of each key
    int nty, ntz;          // tiles along a_2, a_3
    int ntiles;
    int P;                 // key of positions without a cell
    int stall;             // test hook: consumers never release the first stage
};

template <int TZ>
constexpr int stage_rows() { return kCX * kCY * (TZ + 3); }

template <int TZ>
constexpr size_t staged_smem()
{
    return (size_t)TileCfg<TZ>::S * stage_rows<TZ>() * kSlice + sizeof(ElecW) * TileCfg<TZ>::ECAP
         + 2 * TileCfg<TZ>::S * sizeof(uint64_t) + 16;
}

// Warm L2 with size bytes at src (a multiple of 16), without waiting.
__device__ __forceinline__ void prefetch_l2(const void *src, unsigned size)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(size) : "memory");
}


struct TileInfo {
    int x0, y0, z0, nz;
    int start[kTX * kTY], cnt[kTX * kTY];
    int n;
};

template <int TZ>
__device__ __forceinline__ void tile_info(const EvalParams &p, const StagedArgs &a, int t,
                                          TileInfo &ti)
{
    const int bz = t % a.ntz;
    const int r = t / a.ntz;
    const int by = r % a.nty;
    const int bx = r / a.nty;
    ti.x0 = bx * kTX;
    ti.y0 = by * kTY;
    ti.z0 = bz * TZ;
    ti.nz = min(TZ, p.geo.n[2] - ti.z0);
    ti.n = 0;
#pragma unroll
    for (int c = 0; c < kTX * kTY; ++c) {
        const int x = ti.x0 + c / kTY, y = ti.y0 + c % kTY;
        int s = 0, e = 0;
        if (x < p.geo.n[0] && y < p.geo.n[1]) {
            const int k0 = sort_cell_key(p.geo, x, y, ti.z0);     // a_3 runs are consecutive keys
            s = k0 ? a.cell_end[k0 - 1] : 0;
            e = a.cell_end[k0 + ti.nz - 1];
        }
        ti.start[c] = s;
        ti.cnt[c] = e - s;
        ti.n += e - s;
    }
}

// Bounded wait that also gives up once another warp of the CTA has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, unsigned parity,
                                              volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 31u) == 0 && (*abort_flag || global_ns() - t0 > WAIT_LIMIT_NS)) return false;
    }
}

// One warp: geometry and 64 x 5 weights of the electron at tile position q.
template <int TZ>
__device__ __forceinline__ void setup_electron(const EvalParams &p, const TileInfo &ti, int q,
                                               int lane, ElecW &w)
{
    int slot = 0;
    bool found = false;
#pragma unroll
    for (int k = 0; k < kTX * kTY; ++k) {
        if (!found && q < ti.cnt[k]) {
            slot = ti.start[k] + q;
            found = true;
        } else if (!found) {
            q -= ti.cnt[k];
        }
    }
    const int e = p.perm[slot];
    int i0, i1, i2, bad;
    float t0, t1, t2;
    if (p.georec) {
        const int4 gi = *reinterpret_cast<const int4 *>(p.georec + slot);
        const float4 gt = *reinterpret_cast<const float4 *>(&p.georec[slot].t[0]);
        i0 = gi.x; i1 = gi.y; i2 = gi.z; bad = gi.w;
        t0 = gt.x; t1 = gt.y; t2 = gt.z;
    } else {
        int ia = 0;
        float ta = 0.0f;
        bad = 0;
        if (lane < 3) {
            const double *r = p.pos + 3 * (size_t)e;
            bad = wrap_axis(p.geo, lane, r[0], r[1], r[2], ia, ta);
        }
        bad = __reduce_or_sync(FULL, bad);
        i0 = __shfl_sync(FULL, ia, 0); i1 = __shfl_sync(FULL, ia, 1); i2 = __shfl_sync(FULL, ia, 2);
        t0 = __shfl_sync(FULL, ta, 0); t1 = __shfl_sync(FULL, ta, 1); t2 = __shfl_sync(FULL, ta, 2);
    }
    if (lane == 0) {
        // the sort put the electron in this tile, so its cell is inside it;
        // clamp anyway so that shared-memory reads stay in the stage
        const int cx = min(max(i0 - ti.x0, 0), kTX - 1);
        const int cy = min(max(i1 - ti.y0, 0), kTY - 1);
        const int cz = min(max(i2 - ti.z0, 0), TZ - 1);
        w.base = (cx * kCY + cy) * (TZ + 3) + cz;
        w.e = e;
        if (bad) atomicOr(p.status, bad);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int pt = lane + 32 * h;
        site_weights(p.geo, t0, t1, t2, pt, w.w4[pt], w.wl[pt]);
    }
}

// One warp: the 64-site contraction of one electron over one staged chunk.
template <typename T, int TZ, bool VONLY>
__device__ __forceinline__ void contract_electron(const EvalParams &p, const ElecW &w,
                                                  const unsigned char *stage, int chunk, int lane)
{
    constexpr int VEC = Elt<T>::VEC;
    constexpr int NW = VONLY ? 1 : 5;
    float acc[NW][VEC];
#pragma unroll
    for (int k = 0; k < NW; ++k)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[k][v] = 0.0f;
    // the five outputs accumulate in packed pairs of neighbouring elements
    // (same fma per lane as the scalar form, so results are unchanged; half
    // the FMA instructions: measured 6-7 % faster on dense FP32 batches and
    // 9 % more for 16-bit tables than pairs of outputs)
    AccPairs<VEC> ap;
    pairs_zero(ap);
    const unsigned char *sb = stage + (size_t)w.base * kSlice + lane * 16;
    // 16-bit tables keep the a_1 loop rolled: fully unrolled, with the 8-wide
    // unpacking and accumulators, it was measured about 30 % slower
#pragma unroll(sizeof(T) == 4 ? 4 : 1)
    for (int kx = 0; kx < 4; ++kx)
#pragma unroll
        for (int ky = 0; ky < 4; ++ky)
#pragma unroll
            for (int kz = 0; kz < 4; ++kz) {
                const int pt = 16 * kx + 4 * ky + kz;
                const uint4 raw = *reinterpret_cast<const uint4 *>(
                    sb + ((kx * kCY + ky) * (TZ + 3) + kz) * kSlice);
                const float4 ww = w.w4[pt];
                float f[VEC];
                Elt<T>::unpack(raw, f);
                if constexpr (VONLY) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[0][v] = fmaf(ww.x, f[v], acc[0][v]);
                } else {
                    pairs_fma(ap, ww, w.wl[pt], f);
                }
            }
    if constexpr (!VONLY) {
        pairs_out(ap, acc);
    }
    store_chunk<VEC, VONLY>(p, w.e, chunk, lane, acc);
}

template <int CW>
__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(CW * 32) : "memory");
}

template <typename T, int TZ, bool VONLY, int CW>
__global__ void __launch_bounds__(32 * (CW + 1), 1)
    blip_eval_staged(EvalParams p, StagedArgs a, const __grid_constant__ CUtensorMap tmap)
{
    constexpr int VEC = Elt<T>::VEC;
    constexpr int NW = VONLY ? 1 : 5;
    constexpr int kStages = TileCfg<TZ>::S, kECap = TileCfg<TZ>::ECAP;
    constexpr size_t SB = (size_t)stage_rows<TZ>() * kSlice;
    constexpr int kSliceElems = kSlice / (int)sizeof(T);
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *stage0 = smem;
    ElecW *W = reinterpret_cast<ElecW *>(smem + kStages * SB);
    uint64_t *full = reinterpret_cast<uint64_t *>(W + kECap);
    uint64_t *empty = full + kStages;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + kStages);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    check_offsets(p);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, CW);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int n1 = p.geo.n[0], n2 = p.geo.n[1], n3 = p.geo.n[2];
    if (warp == CW) {
        // ---------------- producer ----------------
        const char *tbase = reinterpret_cast<const char *>(p.table);
        const size_t rowb = (size_t)p.row_stride * sizeof(T);
        long long fill = 0;
        bool ok = true;
        TileInfo tn;
        if (blockIdx.x < a.ntiles) tile_info<TZ>(p, a, blockIdx.x, tn);
        for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
            const TileInfo ti = tn;
            // look one tile ahead: its union rows (every chunk) into L2, so
            // that the stage copies of the next tile hit in L2
            if (t + (int)gridDim.x < a.ntiles) {
                tile_info<TZ>(p, a, t + gridDim.x, tn);
                if (tn.n > 0 && lane < kCX * kCY) {
                    const int lx = lane / kCY, ly = lane - lx * kCY;
                    int gx = tn.x0 - 1 + lx, gy = tn.y0 - 1 + ly;
                    gx += gx < 0 ? n1 : 0;
                    gx -= gx >= n1 ? n1 : 0;
                    gy += gy < 0 ? n2 : 0;
                    gy -= gy >= n2 ? n2 : 0;
                    prefetch_l2(tbase + ((size_t)(gx * n2 + gy) * (n3 + 3) + tn.z0) * rowb,
                                (unsigned)((tn.nz + 3) * rowb));
                }
            }
            if (ti.n == 0) continue;
            const int parts = (ti.n + kECap - 1) / kECap;
            for (int part = 0; part < parts && ok; ++part)
                for (int o = 0; o < p.nchunk; ++o) {
                    const int s = (int)(fill % kStages);
                    const long long k = fill / kStages;
                    if (k > 0) {
                        const bool got = wait_or_abort(empty + s, (unsigned)((k - 1) & 1), abort_flag);
                        if (!__all_sync(FULL, got)) {
                            if (lane == 0) {
                                *abort_flag = 1;
                                atomicOr(p.status, BLIP_STATUS_TIMEOUT);
                            }
                            ok = false;
                            break;
                        }
                    }
                    // full boxes of TZ + 3 rows: past the column's last row a box
                    // reads the next column's rows (or zeros past the table),
                    // which no electron of this tile uses
                    if (lane == 0) mbar_expect_tx(full + s, (unsigned)SB);
                    __syncwarp();
                    if (lane < kCX * kCY) {
                        const int col = lane;
                        const int lx = col / kCY, ly = col - lx * kCY;
                        int gx = ti.x0 - 1 + lx, gy = ti.y0 - 1 + ly;
                        gx += gx < 0 ? n1 : 0;
                        gx -= gx >= n1 ? n1 : 0;
                        gy += gy < 0 ? n2 : 0;
                        gy -= gy >= n2 ? n2 : 0;
                        tma_load_2d(stage0 + s * SB + (size_t)col * (TZ + 3) * kSlice, &tmap,
                                    o * kSliceElems, (gx * n2 + gy) * (n3 + 3) + ti.z0, full + s);
                    }
                    ++fill;
                }
        }
        // drain: the copies of the last fills must land before the CTA exits
        for (long long f = fill > kStages ? fill - kStages : 0; f < fill; ++f) {
            const bool got = mbar_wait(full + (int)(f % kStages), (unsigned)((f / kStages) & 1));
            if (!__all_sync(FULL, got) && lane == 0) atomicOr(p.status, BLIP_STATUS_TIMEOUT);
        }
        return;
    }

    // ---------------- consumers ----------------
    const int cw = warp;
    // positions without a cell (last sort bucket): NaN outputs
    {
        const int nan0 = a.cell_end[a.P - 1];
        for (long long sl = nan0 + (long long)blockIdx.x * CW + cw; sl < p.n_elec;
             sl += (long long)gridDim.x * CW) {
            const int e = p.perm[sl];
            if (lane == 0) {
                int bad = BLIP_STATUS_NONFINITE_POS;
                if (p.georec) bad |= p.georec[sl].bad;
                atomicOr(p.status, bad);
            }
            for (int o = 0; o < p.nchunk; ++o) {
                float acc[NW][VEC];
#pragma unroll
                for (int k = 0; k < NW; ++k)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[k][v] = __int_as_float(0x7fc00000);
                store_chunk<VEC, VONLY>(p, e, o, lane, acc);
            }
        }
    }
    long long fill = 0;
    int rot = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        TileInfo ti;
        tile_info<TZ>(p, a, t, ti);
        if (ti.n == 0) continue;
        const int parts = (ti.n + kECap - 1) / kECap;
        for (int part = 0; part < parts; ++part) {
            const int q0 = (int)((long long)part * ti.n / parts);
            const int cnt = (int)((long long)(part + 1) * ti.n / parts) - q0;
            consumer_sync<CW>();   // the previous part's weights are no longer read
            if (!*abort_flag)
                for (int j = cw; j < cnt; j += CW) setup_electron<TZ>(p, ti, q0 + j, lane, W[j]);
            consumer_sync<CW>();
            for (int o = 0; o < p.nchunk; ++o) {
                const int s = (int)(fill % kStages);
                bool have = false;
                if (!*abort_flag) {
                    const bool got = wait_or_abort(full + s, (unsigned)((fill / kStages) & 1), abort_flag);
                    have = __all_sync(FULL, got);
                    if (!have && lane == 0) {
                        *abort_flag = 1;
                        atomicOr(p.status, BLIP_STATUS_TIMEOUT);
                    }
                }
                if (have) {
                    const unsigned char *st = stage0 + s * SB;
                    for (int j = (cw - rot + CW) % CW; j < cnt; j += CW)
                        contract_electron<T, TZ, VONLY>(p, W[j], st, o, lane);
                }
                __syncwarp();
                if (lane == 0 && !(a.stall && fill == 0)) mbar_arrive(empty + s);
                rot = (rot + cnt) % CW;
                ++fill;
            }
        }
    }
}

template <typename T, int TZ, bool VONLY, int CW>
cudaError_t launch_staged_t(const EvalParams &p, StagedArgs a, const CUtensorMap &tmap, int sm_count,
                            cudaStream_t stream)
{
    constexpr size_t smem = staged_smem<TZ>();
    static_assert(smem <= 227 * 1024, "stage ring and weights exceed shared memory");
    static bool attr_set = false;   // raise this instantiation's dynamic shared-memory cap once
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(blip_eval_staged<T, TZ, VONLY, CW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    a.ntz = (p.geo.n[2] + TZ - 1) / TZ;
    a.ntiles = ((p.geo.n[0] + kTX - 1) / kTX) * a.nty * a.ntz;
    const int grid = std::max(1, std::min(sm_count, a.ntiles));
    blip_eval_staged<T, TZ, VONLY, CW><<<grid, 32 * (CW + 1), smem, stream>>>(p, a, tmap);
    return cudaGetLastError();
}

template <typename T, int CW>
cudaError_t launch_staged_cw(const EvalParams &p, const StagedArgs &a, int tz,
                             const CUtensorMap &tm, int sm_count, cudaStream_t stream)
{
    const bool vonly = p.grads == nullptr;
    if (tz == 2)
        return vonly ? launch_staged_t<T, 2, true, CW>(p, a, tm, sm_count, stream)
                     : launch_staged_t<T, 2, false, CW>(p, a, tm, sm_count, stream);
    return vonly ? launch_staged_t<T, 4, true, CW>(p, a, tm, sm_count, stream)
                 : launch_staged_t<T, 4, false, CW>(p, a, tm, sm_count, stream);
}

template <typename T>
cudaError_t launch_staged_elem(const EvalParams &p, const StagedArgs &a, int tz, int cw,
                               const CUtensorMap &tm, int sm_count, cudaStream_t stream)
{
    return cw == 12 ? launch_staged_cw<T, 12>(p, a, tz, tm, sm_count, stream)
                    : launch_staged_cw<T, 16>(p, a, tz, tm, sm_count, stream);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

}  // namespace

static_assert(sizeof(TmaDesc) == sizeof(CUtensorMap), "tensor-map storage size");

cudaError_t make_staged_tmap(const void *table, int elem, long long row_stride, long long rows,
                             int tz, TmaDesc *out)
{
    if ((tz != 2 && tz != 4) || !out || row_stride < 1 || rows < 1) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const CUtensorMapDataType dt = elem == ELEM_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : elem == ELEM_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t esz = elem == ELEM_F32 ? 4 : 2;
    const cuuint64_t dims[2] = {(cuuint64_t)row_stride, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)row_stride * esz};
    const cuuint32_t box[2] = {(cuuint32_t)(kSlice / esz), (cuuint32_t)(tz + 3)};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap *>(out), dt, 2, const_cast<void *>(table), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_staged(const EvalParams &p, int elem, int tz, int cw, const int *cell_end,
                          const TmaDesc &tmap, int sm_count, int stall, cudaStream_t stream)
{
    if ((tz != 2 && tz != 4) || (cw != 12 && cw != 16) || !p.perm || !cell_end || p.n_k)
        return cudaErrorInvalidValue;
    StagedArgs a{};
    a.cell_end = cell_end;
    a.nty = (p.geo.n[1] + kTY - 1) / kTY;
    a.P = (int)sort_key_count(p.geo);
    a.stall = stall;
    const CUtensorMap &tm = *reinterpret_cast<const CUtensorMap *>(&tmap);
    switch (elem) {
    case ELEM_F32: return launch_staged_elem<float>(p, a, tz, cw, tm, sm_count, stream);
    case ELEM_BF16: return launch_staged_elem<__nv_bfloat16>(p, a, tz, cw, tm, sm_count, stream);
    case ELEM_F16: return launch_staged_elem<__half>(p, a, tz, cw, tm, sm_count, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace blip

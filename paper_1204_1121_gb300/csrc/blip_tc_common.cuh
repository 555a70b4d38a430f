// Pieces shared by the two tensor-core kernels (the evaluation kernel of
// blip_tc.cu and the ratio kernel of blip_ratio_tc.cu): the part geometry,
// the work-queue arguments, the tcgen05 / TMA / mbarrier helpers (inline
// PTX) and the walk that cuts a grid column into parts.
#pragma once

#include <cuda.h>
#include <type_traits>

#include "blip_mbar.cuh"

namespace blip {

namespace {

using namespace dev;
using namespace mb;

constexpr int kNE = 25;                 // electrons per part: N = 5 kNE <= 128
constexpr int kSegCells = 5;            // cells along a_3 per part
constexpr int kWin = 8;                 // stored rows per stencil column of a part
constexpr int kCols = 16;               // stencil columns (4 x 4)
constexpr int kK = kCols * kWin;        // 128 union rows = K
constexpr int kMT = 128;                // orbital components per M tile
constexpr int kNmax = 128;
constexpr int kEpiWarps = 8;           // two per tensor-memory lane quarter
constexpr int kThreads = 32 * (2 + kEpiWarps + 4);
constexpr uint32_t kBox = 1024;                          // 8 rows x 128 bytes
constexpr uint32_t kStage = kMT * kK * 2;                // one operand plane of one M tile: 32 KB
constexpr uint32_t kTmemCols = 512;                      // all of tensor memory
constexpr int kColQ = 4;                                 // column ring slots

struct TcArgs {
    const int *cell_end;   // sort: one past the last slot of each key
    const int *cols;       // column keys (key of cell (x, y, 0)) in sort order
    int ncols;
    int P;                 // key of positions without a cell
    int mt;                // M tiles (ceil(Lreal / 128))
    int plane_rows;        // rows of one coefficient plane in the tensor map
    int stall;             // test hook: the MMA thread never releases the first stage
    int wide;              // 1: the 5-D tensor map (8 KB boxes) is usable
    int *col_ctr;          // work queue: the next column to take (0 at launch)
    const float *rcols;    // ratio mode: [n_elec][Lreal] inverse columns, else null
    const float *rsig;     // ratio kernel: per-electron scale of the column operand, or null
    float *ratio;          // ratio mode: [n_elec][5] output, else null
};

// ---------------------------------------------------------------------------
// tcgen05 / TMA helpers (inline PTX)
// ---------------------------------------------------------------------------

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units), the sm_100 descriptor version, swizzle mode.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo,
                                              uint32_t swizzle)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)(swizzle & 7u) << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B of one
// 16-bit type (fmt 0 = FP16, 1 = BF16), A MN-major (a_mn = 1) or K-major
// (a_mn = 0), B K-major, M = 128, N.
__device__ __forceinline__ uint32_t instr_desc(int n, int fmt, uint32_t a_mn = 1u)
{
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | (a_mn << 15) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kMT >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}


// Tiled tensor copy of one 5-D box at element coordinates (c0 .. c4).
__device__ __forceinline__ void tma_load_5d(void *dst, const void *tmap, int c0, int c1, int c2,
                                            int c3, int c4, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void named_sync(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Bounded wait that also gives up once another warp has aborted.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, unsigned parity, volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 31u) == 0 && (*abort_flag || global_ns() - t0 > WAIT_LIMIT_NS)) return false;
    }
}

__device__ __forceinline__ void raise_abort(const EvalParams &p, volatile int *abort_flag)
{
    *abort_flag = 1;
    atomicOr(p.status, BLIP_STATUS_TIMEOUT);
}

// ---------------------------------------------------------------------------
// parts: the same deterministic walk for the producer and the weight warps
// ---------------------------------------------------------------------------

// Cell counts of one grid column, read by a whole warp: lane i holds
// cell_end[k0 + base + i] (one coalesced load per 32 cells), and the walk
// reads them by shuffle, so the part walk has no chain of dependent loads.
struct ColumnEnds {
    int k0, base, val;
};

__device__ __forceinline__ void ends_init(const TcArgs &a, int k0, int n3, int lane, ColumnEnds &w)
{
    w.k0 = k0;
    w.base = 0;
    w.val = lane < n3 ? a.cell_end[k0 + lane] : 0;
}

// cell_end[k0 + z]; every lane of the warp calls it with the same z
__device__ __forceinline__ int ends_at(const TcArgs &a, int n3, int lane, ColumnEnds &w, int z)
{
    if (z < w.base || z >= w.base + 32) {
        w.base = z;
        w.val = z + lane < n3 ? a.cell_end[w.k0 + z + lane] : 0;
    }
    return __shfl_sync(FULL, w.val, z - w.base);
}

struct Cursor {
    int z;        // current cell along a_3
    int used;     // electrons of cell z already in earlier parts
    int sbase;    // first slot of cell z
};

__device__ __forceinline__ void cursor_init(const TcArgs &a, int k0, Cursor &c)
{
    c.z = 0;
    c.used = 0;
    c.sbase = k0 ? a.cell_end[k0 - 1] : 0;
}

// Next part of the column: up to kNE electrons from at most kSegCells
// consecutive cells, starting at the first cell with electrons left; a cell
// with more than kNE electrons gives parts of kNE of its own.  Returns false
// when the column is done.  Called by every lane of a warp alike.
__device__ __forceinline__ bool next_part(const TcArgs &a, int n3, int lane, ColumnEnds &w,
                                          Cursor &c, int &z0, int &s0, int &cnt)
{
    for (;;) {
        if (c.z >= n3) return false;
        const int end = ends_at(a, n3, lane, w, c.z);
        if (end - c.sbase - c.used > 0) break;
        c.sbase = end;
        c.used = 0;
        ++c.z;
    }
    z0 = c.z;
    s0 = c.sbase + c.used;
    const int end0 = ends_at(a, n3, lane, w, c.z);
    if (end0 - s0 >= kNE) {
        cnt = kNE;
        c.used += kNE;
        return true;
    }
    cnt = end0 - s0;
    c.sbase = end0;
    c.used = 0;
    ++c.z;
    while (c.z < n3 && c.z < z0 + kSegCells) {
        const int e = ends_at(a, n3, lane, w, c.z);
        if (cnt + (e - c.sbase) > kNE) break;
        cnt += e - c.sbase;
        c.sbase = e;
        ++c.z;
    }
    return true;
}

__device__ __forceinline__ void column_xy(const Geometry &g, int k0, int &x, int &y)
{
    // invert sort_cell_key(x, y, 0) = ((sb * 16 + br) * 64 + col) * n3
    const int q = k0 / g.n[2];
    const int col = q & 63, br = (q >> 6) & 15, sb = q >> 10;
    const int nsy = (g.n[1] + 31) >> 5;
    x = (sb / nsy) * 32 + (br >> 2) * 8 + (col >> 3);
    y = (sb % nsy) * 32 + (br & 3) * 8 + (col & 7);
}

// Bit pattern of a 16-bit value of type T.
template <typename T> __device__ __forceinline__ unsigned short to_bits(float v);
template <> __device__ __forceinline__ unsigned short to_bits<__nv_bfloat16>(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <> __device__ __forceinline__ unsigned short to_bits<__half>(float v)
{
    return __half_as_ushort(__float2half_rn(v));
}
// Two FP32 values as one packed pair of T (round to nearest; a in the low
// half), and a packed pair back to FP32.
template <typename T> __device__ __forceinline__ uint32_t pack2(float a, float b);
template <> __device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}
template <> __device__ __forceinline__ uint32_t pack2<__half>(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}
template <typename T> __device__ __forceinline__ float2 unpack2(uint32_t w);
template <> __device__ __forceinline__ float2 unpack2<__nv_bfloat16>(uint32_t w)
{
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <> __device__ __forceinline__ float2 unpack2<__half>(uint32_t w)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
template <typename T> __device__ __forceinline__ float from_bits(unsigned short b);
template <> __device__ __forceinline__ float from_bits<__nv_bfloat16>(unsigned short b)
{
    return __bfloat162float(__ushort_as_bfloat16(b));
}
template <> __device__ __forceinline__ float from_bits<__half>(unsigned short b)
{
    return __half2float(__ushort_as_half(b));
}

// 16 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// 8 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace

}  // namespace blip

// Tensor-core evaluation kernel for dense sorted batches (variant 12).
//
// When a quasi-simultaneous batch (Sec. IV.A) holds many electrons per grid
// cell, the electrons of a few neighbouring cells share their stencil rows
// (Eq. 7), and the contraction of Eq. 11.12.24.1 over those rows becomes a
// dense matrix product.  A part is up to kNE electrons from at most 5
// consecutive cells along a_3 of one grid column (x, y); every stencil of
// the part lies in the union of 16 stencil columns (x - 1 .. x + 2,
// y - 1 .. y + 2) x 8 stored rows (z0 .. z0 + 7, the ghost-plane layout).
// With K = 128 union rows:
//
//     D^T[l][(j, o)] = sum_k  a[k][l]  W_o^{(j)}[k]
//
// M = 128 orbital components per tile (the stored rows, orbital-contiguous,
// are the MN-major A operand as they stand), N = 5 x electrons (value,
// d/dx, d/dy, d/dz, Laplacian weights of each electron, zero outside its 64
// sites; the K-major B operand, built on the chip).  The weights are split
// into two 16-bit parts (hi + lo, the same type as the table) so the
// weight rounding is about 2^-17 relative; the coefficients enter as stored.
// FP32 tables enter as two FP16 planes of a / s_l (s_l a power of two at or
// above the component's largest |a|, so the division is exact): hi = RN(a /
// s_l), lo = RN(a / s_l - hi), 22 significant bits; with FP16 weights split
// the same way, three products per K step (hi.hi, hi.lo, lo.hi) leave out
// lo.lo, below 2^-22 relative; s_l is applied in the epilogue.  Products are
// accumulated in FP32 in tensor memory.
//
// Persistent grid, one CTA per SM, 14 warps; the CTAs take grid columns
// from a work queue (a global counter over the columns in sort order):
//   warp 0      takes the columns (skipping empty ones) and passes them to
//               the weight warps through a 4-slot ring; TMA producer: per
//               (part, M tile, plane) the 16 stencil
//               columns x 2 halves of 8 rows x 64 components into a 3-stage
//               ring, as 4 boxes of 8 KB (4 consecutive grid columns x 2
//               halves, a 5-D view of the table) or, where the columns wrap
//               around the cell, 32 boxes of 1 KB;
//   warp 1      allocates tensor memory and issues the MMAs (one thread):
//               per M tile, 8 K steps x planes products into one of the
//               FP32 accumulators (two of 256 columns, four of 64 for
//               values only), then tcgen05.commit to the stage's empty
//               barrier and the accumulator's full barrier;
//   warps 2-9   epilogue, two warps per lane quarter of the accumulator:
//               tensor memory -> registers (tcgen05.ld), scale, streaming
//               stores through a per-column output-row pointer (a warp
//               writes 32 consecutive components of one output);
//   warps 10-13 weights: the part's electrons (geometry from the sort's
//               per-slot records, or the FP64 wrap), their 64 x 5 weights
//               split into 16-bit planes, written as B operand core
//               matrices into one of two buffers.
// Ratio mode (blip_eval_ratio): the epilogue contracts the accumulator
// columns with the inverse Slater column of each electron instead of storing
// them, sum_l D^T[l][(j, o)] c_j[l] (the quasi-simultaneous ratio and its
// derivatives): per lane over the M tiles of a part, then over the 32 lanes
// (a fixed butterfly that leaves each lane two column totals), then over the
// four lane quarters in shared memory (the part's weight buffer, free once
// its last product is done), in a fixed order; five numbers per electron
// leave the chip (plus the new orbital row if asked for).
// Every wait is bounded (about 2 s of global time): a wait that runs out
// sets BLIP_STATUS_TIMEOUT and an abort flag; every role then winds down,
// the producer waits (bounded) for its copies in flight and the MMA thread
// for its products before the tensor memory is freed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "blip_tc_common.cuh"

namespace blip {

namespace {

using namespace dev;
using namespace mb;

// Shapes of one instantiation: APL coefficient planes per M tile (1: the
// 16-bit table as stored; 2: an FP32 table as two FP16 planes, hi + lo, of
// the coefficient over a power-of-two per-component scale); the weights in
// two 16-bit parts stacked along N in one B operand (rows [0, RLO) the hi
// part of the part's NO x cnt rows, rows [RLO, 2 RLO) the lo part; RLO = 128
// with five outputs, 32 values only), so that one product of N = RLO + NH
// covers both (an M = 128, K = 16 product costs the same for any N up to
// 256: measured 150 cycles); two buffers of it (the next part's weights are
// built while the current part's products run); as many 32 KB operand
// stages as the rest of shared memory holds; accumulators of 2 RLO columns
// (hi, then lo products), as many as tensor memory holds (at most 4).
template <int APL, bool VONLY> struct TcCfg {
    static constexpr int RLO = VONLY ? 32 : kNmax;
    static constexpr int WROWS = 2 * RLO;
    static constexpr uint32_t KGROUP = WROWS * 16;           // bytes per K group (8 rows of K)
    static constexpr uint32_t W_BUF = KGROUP * kCols;        // the stacked B operand
    static constexpr int WB = 2;
    static constexpr int STAGES = (int)((229376u - WB * W_BUF) / kStage);
    static constexpr int ACC_COLS = 2 * RLO;
    static constexpr int NACC = (int)(kTmemCols / ACC_COLS) > 4 ? 4 : (int)(kTmemCols / ACC_COLS);
};

// Part bookkeeping shared by the weight warps (writers), the MMA thread and
// the epilogue (readers), one per weight buffer.
struct __align__(16) PartInfo {
    int cnt;            // electrons, or -1 for "no more parts"
    int n;              // MMA N: outputs x cnt rounded up to 16
    int pad[2];
    float *dst[kNmax];  // output row of accumulator column NO j + o (electron j, output o)
    int eid[32];        // ratio mode: electron index of part electron j
};


template <int APL, bool VONLY>
constexpr size_t tc_smem()
{
    using C = TcCfg<APL, VONLY>;
    return C::STAGES * kStage + C::WB * C::W_BUF + 2 * sizeof(PartInfo) + 512;
}

// Epilogue of the ratio mode for one warp: lane quarter q of the
// accumulator, the 32-column chunks c0 = 32 HALF + 64 i (i = 0, 1) of the
// part's 5 cnt columns (electron j = column / 5, output o = column % 5).
// Per M tile each lane folds its orbital component l into 64 running sums,
// sum over tiles of (hi + lo weight part columns) s_l c_j[l]; at the
// end of the part a butterfly over the lanes leaves lane L the totals of its
// chunk columns 2 L and 2 L + 1, the four quarters meet in the part's weight
// buffer, and thread et < 5 cnt of the epilogue writes
// ratio[e_j][o] = q0 + q1 + q2 + q3 (this order).  Returns false on abort.
template <int HALF, int RLO, int ACC_COLS, int NACC>
__device__ __forceinline__ bool ratio_epilogue(const EvalParams &p, const TcArgs &a,
                                               PartInfo *info, unsigned char *wbuf,
                                               uint32_t w_buf_bytes, uint64_t *w_full,
                                               uint64_t *acc_full, uint64_t *acc_empty,
                                               uint64_t *epi_done, uint64_t *red_done,
                                               uint32_t tmem, int q, int lane, int et,
                                               volatile int *abort_flag)
{
    const size_t L = (size_t)p.Lreal;
    int tile = 0;
    for (int part = 0;; ++part) {
        const int wi = (int)(part & 1);
        const unsigned ph = (unsigned)((part >> 1) & 1);
        if (!wait_bar(w_full + wi, ph, abort_flag)) {
            if (lane == 0) raise_abort(p, abort_flag);
            return false;
        }
        const int cnt = info[wi].cnt;
        if (cnt < 0) return true;
        const int ncol = 5 * cnt;
        const int *eid = info[wi].eid;
        float acc[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) acc[i] = 0.0f;
        for (int m = 0; m < a.mt; ++m) {
            const int ab = (int)(tile % NACC);
            const int l = m * kMT + 32 * q + lane;
            const bool in = l < p.Lreal;
            const float sc = (p.scales && in) ? p.scales[l] : 1.0f;
            // s_l c_j[l] of the chunks' electrons, loaded ahead of the
            // accumulator (each inverse entry is read once: streaming loads)
            float cv[2][8];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int c0 = 32 * HALF + 64 * i;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = c0 / 5 + u;
                    cv[i][u] = (in && j <= (c0 + 31) / 5 && j < cnt)
                                   ? __ldcs(a.rcols + (size_t)eid[j] * L + l) * sc
                                   : 0.0f;
                }
            }
            if (!wait_bar(acc_full + ab, (unsigned)((tile / NACC) & 1), abort_flag)) {
                if (lane == 0) raise_abort(p, abort_flag);
                return false;
            }
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * ACC_COLS);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int c0 = 32 * HALF + 64 * i;
                if (c0 >= ncol) break;                   // the same for the whole warp
#pragma unroll
                for (int g = 0; g < 4; ++g) {            // 8 columns at a time
                    uint32_t r[8], rl[8];
                    tmem_ld8_nowait(taddr + c0 + 8 * g, r);              // hi weight part
                    tmem_ld8_nowait(taddr + RLO + c0 + 8 * g, rl);       // lo weight part
                    tmem_wait_ld();
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const int cc = c0 + 8 * g + jj, u = cc / 5 - c0 / 5;
                        if (cc < ncol) {
                            const float v = __uint_as_float(r[jj]) + __uint_as_float(rl[jj]);
                            acc[32 * i + 8 * g + jj] = fmaf(v, cv[i][u], acc[32 * i + 8 * g + jj]);
                            if (cc % 5 == 0 && p.values && in)
                                __stcs(p.values + (size_t)eid[cc / 5] * L + l, v * sc);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + ab);
            ++tile;
        }
        // over the lanes: after the step with offset o the lanes with bit o
        // set keep the upper half of the sums in play
#pragma unroll
        for (int st = 0; st < 5; ++st) {
            const int o = 16 >> st, h = 32 >> st;
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float send = up ? acc[i] : acc[i + h];
                const float keep = up ? acc[i + h] : acc[i];
                acc[i] = keep + __shfl_xor_sync(FULL, send, o);
            }
        }
        // the part's weight buffer is free: its last product has completed
        float *scr = reinterpret_cast<float *>(wbuf + (uint32_t)wi * w_buf_bytes);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int k = 2 * lane + t;
            scr[q * 128 + 32 * HALF + 64 * (k >> 5) + (k & 31)] = acc[t];
        }
        mbar_arrive(red_done + wi);                      // all 32 kEpiWarps threads
        if (!wait_bar(red_done + wi, ph, abort_flag)) {
            if (lane == 0) raise_abort(p, abort_flag);
            return false;
        }
        if (et < ncol) {
            const float tot = ((scr[et] + scr[128 + et]) + scr[256 + et]) + scr[384 + et];
            a.ratio[(size_t)eid[et / 5] * 5 + et % 5] = tot;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(epi_done + wi);
    }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

// T: the 16-bit operand type; APL: coefficient planes (1: the 16-bit table;
// 2: an FP32 table as two scaled FP16 planes); MODE: 0 the five outputs,
// 1 values only, 2 the ratio contraction.
template <typename T, int APL, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    blip_eval_tc(EvalParams p, TcArgs a, const __grid_constant__ CUtensorMap tmap,
                 const __grid_constant__ CUtensorMap tmap5)
{
    constexpr bool VONLY = MODE == 1;
    using Cfg = TcCfg<APL, VONLY>;
    constexpr int WPL = 2, WB = Cfg::WB, NS = Cfg::STAGES;    // WPL: weight parts (hi, lo)
    constexpr int NO = VONLY ? 1 : 5;                    // outputs per electron
    constexpr int FMT = std::is_same<T, __nv_bfloat16>::value ? 1 : 0;
    extern __shared__ __align__(1024) unsigned char smem[];
    // the 128-byte-swizzled operand stages need 1024-byte alignment: give up
    // (status bit, no output) if the dynamic shared memory does not have it
    if (smem_addr(smem) & 1023u) {
        if (threadIdx.x == 0) atomicOr(p.status, BLIP_STATUS_LAYOUT);
        return;
    }
    unsigned char *stageA = smem;
    unsigned char *wbuf = smem + NS * kStage;
    PartInfo *info = reinterpret_cast<PartInfo *>(wbuf + WB * Cfg::W_BUF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(info + 2);
    uint64_t *a_full = bars, *a_empty = bars + NS;
    uint64_t *w_full = bars + 2 * NS, *w_empty = w_full + 2, *epi_done = w_full + 4;
    constexpr int kAcc = Cfg::NACC;
    uint64_t *acc_full = w_full + 6, *acc_empty = acc_full + kAcc, *drain = acc_empty + kAcc;
    uint64_t *red_done = drain + 1;
    uint64_t *cq_full = red_done + 2, *cq_empty = cq_full + kColQ;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(cq_empty + kColQ);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *colq = abort_flag + 1;           // the column ring
    volatile int *decision = colq + kColQ;         // weight warps: 1 = stop

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n2 = p.geo.n[1], n3 = p.geo.n[2];
    check_offsets(p);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(a_full + s, 1);
            mbar_init(a_empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(w_full + b, 1);
            mbar_init(w_empty + b, 1);
            mbar_init(epi_done + b, kEpiWarps);
            mbar_init(red_done + b, 32 * kEpiWarps);
        }
        for (int b = 0; b < kAcc; ++b) {
            mbar_init(acc_full + b, 1);
            mbar_init(acc_empty + b, kEpiWarps);
        }
        mbar_init(drain, 1);
        for (int q = 0; q < kColQ; ++q) {
            mbar_init(cq_full + q, 1);
            mbar_init(cq_empty + q, 4);              // the four weight warps
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        long long fill = 0;
        bool ok = true;
        // stage layout: stencil column (kx, ky), component half h at
        // kx 8 KB + h 4 KB + ky 1 KB (one 128-byte-swizzled 8-row atom each)
        const int c = lane >> 1, h = lane & 1;     // narrow boxes: column c, half h
        const int kxl = c >> 2, kyl = c & 3;
        // Columns come from a work queue shared by the CTAs (a global counter,
        // so the CTAs stay on neighbouring columns in sort order and each
        // takes more as it finishes); each taken column goes into the ring
        // for the weight warps, two columns ahead of this warp's own use
        // (the weight warps run at most two parts ahead of it).
        int pushed = 0;
        bool more = true;
        auto push = [&]() -> int {                   // column, -1 at the end, -2 on abort
            if (!more) return -1;
            const int slot = pushed % kColQ;
            if (pushed >= kColQ) {
                const bool got = wait_bar(cq_empty + slot, (unsigned)(((pushed / kColQ) - 1) & 1),
                                          abort_flag);
                if (!__all_sync(FULL, got)) {
                    if (lane == 0) raise_abort(p, abort_flag);
                    return -2;
                }
            }
            int col = 0;
            if (lane == 0) {
                // columns without electrons are skipped here, so every column
                // in the ring has a part: the weight warps, at most two parts
                // ahead of this warp, never wait for a column it has not pushed
                for (;;) {
                    col = atomicAdd(a.col_ctr, 1);
                    if (col >= a.ncols) break;
                    const int kc = a.cols[col];
                    if (a.cell_end[kc + n3 - 1] > (kc ? a.cell_end[kc - 1] : 0)) break;
                }
                colq[slot] = col < a.ncols ? col : -1;
                mbar_arrive(cq_full + slot);
            }
            col = __shfl_sync(FULL, col, 0);
            ++pushed;
            if (col >= a.ncols) {
                more = false;
                return -1;
            }
            return col;
        };
        int q0 = push(), q1 = push();
        ok = q0 != -2 && q1 != -2;
        while (ok && q0 >= 0) {
            const int q2 = push();
            if (q2 == -2) break;
            const int ci = q0;
            q0 = q1;
            q1 = q2;
            const int k0 = a.cols[ci];
            int x, y;
            column_xy(p.geo, k0, x, y);
            // the 4 stencil columns y - 1 .. y + 2 of one kx are consecutive in
            // memory unless they wrap around the cell: then one 8 KB box per kx
            // (5-D view), else 1 KB boxes
            const bool wide = a.wide && y >= 1 && y + 2 < n2;
            int gx = x - 1 + (wide ? lane : kxl), gy = y - 1 + kyl;
            gx += gx < 0 ? p.geo.n[0] : 0;
            gx -= gx >= p.geo.n[0] ? p.geo.n[0] : 0;
            gy += gy < 0 ? n2 : 0;
            gy -= gy >= n2 ? n2 : 0;
            const int colrow = (gx * n2 + gy) * (n3 + 3);
            Cursor cur;
            cursor_init(a, k0, cur);
            ColumnEnds ends;
            ends_init(a, k0, n3, lane, ends);
            int z0, s0, cnt;
            while (ok && next_part(a, n3, lane, ends, cur, z0, s0, cnt)) {
                for (int m = 0; m < a.mt && ok; ++m)
                    for (int pl = 0; pl < APL; ++pl) {           // FP32: hi, then lo
                        const int s = (int)(fill % NS);
                        const long long k = fill / NS;
                        if (k > 0) {
                            const bool got = wait_bar(a_empty + s, (unsigned)((k - 1) & 1), abort_flag);
                            if (!__all_sync(FULL, got)) {
                                if (lane == 0) raise_abort(p, abort_flag);
                                ok = false;
                                break;
                            }
                        }
                        if (lane == 0) mbar_expect_tx(a_full + s, kStage);
                        __syncwarp();
                        unsigned char *st = stageA + s * kStage;
                        if (wide) {
                            if (lane < 4)
                                tma_load_5d(st + lane * 8192, &tmap5, 0, z0, gx * n2 + y - 1, 2 * m, pl,
                                            a_full + s);
                        } else {
                            tma_load_2d(st + kxl * 8192 + h * 4096 + kyl * kBox, &tmap,
                                        m * kMT + 64 * h, pl * a.plane_rows + colrow + z0, a_full + s);
                        }
                        ++fill;
                    }
            }
        }
        // drain: the copies of the last fills must land before the CTA exits
        for (long long f = fill > NS ? fill - NS : 0; f < fill; ++f) {
            const bool got = mbar_wait(a_full + (int)(f % NS), (unsigned)((f / NS) & 1));
            if (!__all_sync(FULL, got) && lane == 0) atomicOr(p.status, BLIP_STATUS_TIMEOUT);
        }
    } else if (warp == 1) {
        // ---------------- MMA issue (one thread) ----------------
        // lane 0 alone: no warp votes or warp barriers between the products
        // of consecutive stages, so the tensor pipe's short queue stays fed
        if (lane == 0) {
            // A single thread runs this loop, so every instruction's latency
            // counts: ring positions and parities are kept incrementally, and
            // the descriptors are those of stage 0 / weight buffer 0 plus the
            // byte offset / 16 (the 14-bit address field cannot carry: shared
            // addresses stay below 2^18)
            bool ok = true, first = true;
            int s = 0, s_ph = 0;                     // stage ring slot, its fill parity
            int ab = 0, ab_ph = 0, tiles = 0;        // accumulator slot, its round parity
            const uint64_t a_desc0 = smem_desc(smem_addr(stageA), 4096u, kBox, 2);
            const uint64_t b_desc0 = smem_desc(smem_addr(wbuf), Cfg::KGROUP, 128u, 0);
            for (int part = 0; ok; ++part) {
                const int wi = part & 1;                         // info slot
                const int wb = WB == 2 ? wi : 0;                 // weight buffer
                if (!wait_bar(w_full + wi, (unsigned)((part >> 1) & 1), abort_flag)) {
                    raise_abort(p, abort_flag);
                    break;
                }
                if (info[wi].cnt < 0) break;
                const int nh = info[wi].n;                       // rows of one weight part
                const uint32_t id_both = instr_desc(Cfg::RLO + nh, FMT);   // hi and lo parts
                const uint32_t id_hi = instr_desc(nh, FMT);                 // hi part only
                const uint64_t bd0 = b_desc0 + (uint64_t)((wb * Cfg::W_BUF) >> 4);
                for (int m = 0; m < a.mt && ok; ++m) {
                    if (tiles >= kAcc &&
                        !wait_bar(acc_empty + ab, (unsigned)(ab_ph ^ 1), abort_flag)) {
                        raise_abort(p, abort_flag);
                        ok = false;
                        break;
                    }
                    const uint32_t d = tmem + (uint32_t)(ab * Cfg::ACC_COLS);
                    // the hi plane first: its product (N = RLO + NH) sets every
                    // column the epilogue reads; the lo plane's (N = NH) adds
                    for (int pl = 0; pl < APL; ++pl) {
                        if (!wait_bar(a_full + s, (unsigned)s_ph, abort_flag)) {
                            raise_abort(p, abort_flag);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad0 = a_desc0 + (uint64_t)((s * kStage) >> 4);
                        // a 16-bit table (pl = 0) meets both weight parts in one
                        // product; of an FP32 table's planes the lo one meets the
                        // hi weights only (lo x lo is below 2^-22 relative)
                        const uint32_t id = (APL == 2 && pl == 1) ? id_hi : id_both;
#pragma unroll
                        for (int ks = 0; ks < kK / 16; ++ks) {
                            // A: K step ks = stencil columns (kx, ky), (kx, ky + 1)
                            // with kx = ks / 2, ky = 2 (ks % 2): 1 KB apart, the
                            // second 64-component half 4 KB on; B: K groups of 8
                            // at KGROUP bytes, N groups of 8 rows at 128 B
                            const uint64_t ad =
                                ad0 + (uint64_t)(((ks >> 1) * 8192 + (ks & 1) * 2 * kBox) >> 4);
                            const uint64_t bd = bd0 + (uint64_t)((ks * 2 * Cfg::KGROUP) >> 4);
                            mma_f16(d, ad, bd, id, (pl == 0 && ks == 0) ? 0u : 1u);
                        }
                        if (!(a.stall && first)) mma_commit(a_empty + s);
                        first = false;
                        if (pl == APL - 1) {
                            mma_commit(acc_full + ab);
                            if (m == a.mt - 1) mma_commit(w_empty + wi);
                        }
                        if (++s == NS) {
                            s = 0;
                            s_ph ^= 1;
                        }
                    }
                    if (ok) {
                        ++tiles;
                        if (++ab == kAcc) {
                            ab = 0;
                            ab_ph ^= 1;
                        }
                    }
                }
            }
            // every product issued (also those of a tile cut short by an abort)
            // must be done before the tensor memory is freed
            mma_commit(drain);
            if (!mbar_wait(drain, 0)) atomicOr(p.status, BLIP_STATUS_TIMEOUT);
        }
        __syncwarp();
    } else if (warp < 2 + kEpiWarps) {
        // ---------------- epilogue ----------------
        // warps 2 .. 9: lane quarter q = warp % 4 of the accumulator; the two
        // warps of a quarter take alternate 32-column chunks
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const int et = threadIdx.x - 64;             // 0 .. 32 kEpiWarps - 1
        const size_t L = (size_t)p.Lreal;
        // positions without a cell (last sort bucket): NaN outputs
        {
            const int nan0 = a.cell_end[a.P - 1];
            const float nan = __int_as_float(0x7fc00000);
            for (int sl = nan0; sl < p.n_elec; ++sl) {
                if ((sl - nan0) % (int)gridDim.x != (int)blockIdx.x) continue;
                const size_t e = (size_t)p.perm[sl];
                if (et == 0) {
                    int bad = BLIP_STATUS_NONFINITE_POS;
                    if (p.georec) bad |= p.georec[sl].bad;
                    atomicOr(p.status, bad);
                }
                if (MODE == 2 && et < 5) a.ratio[e * 5 + et] = nan;
                for (int l = et; l < p.Lreal; l += 32 * kEpiWarps) {
                    if (MODE == 2) {
                        if (p.values) p.values[e * L + l] = nan;
                        continue;
                    }
                    p.values[e * L + l] = nan;
                    if (!VONLY) {
                        p.grads[e * 3 * L + l] = nan;
                        p.grads[e * 3 * L + L + l] = nan;
                        p.grads[e * 3 * L + 2 * L + l] = nan;
                        p.laps[e * L + l] = nan;
                    }
                }
            }
        }
        if constexpr (MODE == 2) {
            if (half == 0)
                ratio_epilogue<0, Cfg::RLO, Cfg::ACC_COLS, kAcc>(
                    p, a, info, wbuf, Cfg::W_BUF, w_full, acc_full, acc_empty, epi_done, red_done,
                    tmem, q, lane, et, abort_flag);
            else
                ratio_epilogue<1, Cfg::RLO, Cfg::ACC_COLS, kAcc>(
                    p, a, info, wbuf, Cfg::W_BUF, w_full, acc_full, acc_empty, epi_done, red_done,
                    tmem, q, lane, et, abort_flag);
        }
        long long tile = 0;
        for (long long part = 0; MODE != 2; ++part) {
            const int wi = (int)(part & 1);
            if (!wait_bar(w_full + wi, (unsigned)((part >> 1) & 1), abort_flag)) {
                if (lane == 0) raise_abort(p, abort_flag);
                break;
            }
            const int cnt = info[wi].cnt;
            if (cnt < 0) break;
            float *const *dst = info[wi].dst;
            const int ncol = NO * cnt;
            bool ok = true;
            for (int m = 0; m < a.mt; ++m) {
                const int ab = (int)(tile % kAcc);
                if (!wait_bar(acc_full + ab, (unsigned)((tile / kAcc) & 1), abort_flag)) {
                    if (lane == 0) raise_abort(p, abort_flag);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int l = m * kMT + 32 * q + lane;
                const bool in = l < p.Lreal;
                const float sc = (p.scales && in) ? p.scales[l] : 1.0f;
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) +
                                       (uint32_t)(ab * Cfg::ACC_COLS);
                for (int c0 = 32 * half; c0 < ncol; c0 += 64) {
                    // the hi-part products in column c, the lo-part ones RLO on
                    uint32_t r[32], rl[32];
                    tmem_ld32_nowait(taddr + c0, r);
                    tmem_ld32_nowait(taddr + Cfg::RLO + c0, rl);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (in) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj)
                            if (c0 + jj < ncol)
                                __stcs(dst[c0 + jj] + l,
                                       (__uint_as_float(r[jj]) + __uint_as_float(rl[jj])) * sc);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty + ab);
                ++tile;
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(epi_done + wi);
        }
    } else {
        // ---------------- weights ----------------
        // lane j = electron j of the part; weight warp ww writes the 4 stencil
        // columns (kx, ky = ww), kx = 0..3.  Row r = NO j + o of the B operand
        // (plus RLO for the lo part) sits 16 r bytes into a column's K group,
        // so the 32 lanes of a store hit 32 different 16-byte slots (stride 80
        // or 16 bytes): no bank conflicts.
        const int ww = warp - 2 - kEpiWarps;
        bool ok = true;
        long long part = 0;
        // the info slot (and weight buffer) of a part is reused once the MMA
        // thread and the epilogue have released the part that used it last
        auto claim = [&]() -> bool {
            const int wi = (int)(part & 1);
            bool got = true;
            if (part >= 2) {
                const unsigned ph = (unsigned)(((part >> 1) - 1) & 1);
                got = wait_bar(w_empty + wi, ph, abort_flag);
                if (got) got = wait_bar(epi_done + wi, ph, abort_flag);
            }
            if (got && WB == 1 && part >= 1) {
                // one weight buffer: the previous part's products must be done
                const long long pp = part - 1;
                got = wait_bar(w_empty + (int)(pp & 1), (unsigned)((pp >> 1) & 1), abort_flag);
            }
            if (!__all_sync(FULL, got) && lane == 0) raise_abort(p, abort_flag);
            // one thread reads the abort flag between two barriers, so the four
            // warps take the same decision (and meet the same barriers after it)
            named_sync(1, 128);
            if (ww == 0 && lane == 0) *decision = *abort_flag;
            named_sync(1, 128);
            return !*decision;
        };
        const float *J = p.geo.J, *M = p.geo.M;
        const float nrm = p.geo.norm;
        // the parts of this CTA's columns in order, one part ahead: the next
        // part's electron records are loaded while this part's weights are
        // built (their latency was the weight warps' main cost)
        int taken = 0;
        auto take = [&]() -> int {                   // the producer's next column, -1 at the end
            const int slot = taken % kColQ;
            const bool got = wait_bar(cq_full + slot, (unsigned)((taken / kColQ) & 1), abort_flag);
            if (!__all_sync(FULL, got)) {
                if (lane == 0) raise_abort(p, abort_flag);
                return -1;
            }
            const int col = colq[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(cq_empty + slot);
            ++taken;
            return col;
        };
        int ci = take();
        Cursor cur;
        ColumnEnds ends;
        if (ci >= 0) {
            cursor_init(a, a.cols[ci], cur);
            ends_init(a, a.cols[ci], n3, lane, ends);
        }
        auto advance = [&](int &z0_, int &s0_, int &cnt_) -> bool {
            while (ci >= 0) {
                if (next_part(a, n3, lane, ends, cur, z0_, s0_, cnt_)) return true;
                ci = take();
                if (ci >= 0) {
                    cursor_init(a, a.cols[ci], cur);
                    ends_init(a, a.cols[ci], n3, lane, ends);
                }
            }
            return false;
        };
        struct Rec {
            int e;
            int4 gi;
            float4 gt;
        };
        auto load_rec = [&](int s0_, int cnt_, Rec &r) {
            if (lane < cnt_) {
                const int slot = s0_ + lane;
                r.e = p.perm[slot];
                if (p.georec) {
                    r.gi = *reinterpret_cast<const int4 *>(p.georec + slot);
                    r.gt = *reinterpret_cast<const float4 *>(&p.georec[slot].t[0]);
                }
            }
        };
        int nz0 = 0, ns0 = 0, ncnt = 0;
        Rec nrec{};
        bool have = advance(nz0, ns0, ncnt);
        if (have) load_rec(ns0, ncnt, nrec);
        while (have && ok) {
            const int z0 = nz0, cnt = ncnt;
            const Rec rec = nrec;
            have = advance(nz0, ns0, ncnt);
            if (have) load_rec(ns0, ncnt, nrec);
            {
                if (!claim()) {
                    ok = false;
                    break;
                }
                const int wi = (int)(part & 1);
                const int wb = WB == 2 ? wi : 0;
                const int N = (NO * cnt + 15) & ~15;
                const int j = lane;
                // this lane's electron: geometry, 1-D factors
                int cz = 0;
                float X[4][3], Y[3], Z[4][3];
                if (j < cnt) {
                    const int e = rec.e;
                    int i2, bad;
                    float t0, t1, t2;
                    if (p.georec) {
                        i2 = rec.gi.z;
                        bad = rec.gi.w;
                        t0 = rec.gt.x;
                        t1 = rec.gt.y;
                        t2 = rec.gt.z;
                    } else {
                        const double *rp = p.pos + 3 * (size_t)e;
                        int i0, i1;
                        bad = wrap_axis(p.geo, 0, rp[0], rp[1], rp[2], i0, t0);
                        bad |= wrap_axis(p.geo, 1, rp[0], rp[1], rp[2], i1, t1);
                        bad |= wrap_axis(p.geo, 2, rp[0], rp[1], rp[2], i2, t2);
                    }
                    // the sort put the electron in one of the part's cells; clamp
                    // anyway so that every weight stays inside its 8-row window
                    cz = min(max(i2 - z0, 0), kSegCells - 1);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        bspline_1d(t0, k, X[k][0], X[k][1], X[k][2]);
                        bspline_1d(t2, k, Z[k][0], Z[k][1], Z[k][2]);
                    }
                    bspline_1d(t1, ww, Y[0], Y[1], Y[2]);
                    if (ww == 0) {
                        if (bad) atomicOr(p.status, bad);
                        float **dst = info[wi].dst;
                        const size_t L = (size_t)p.Lreal;
                        if constexpr (MODE == 2) {
                            info[wi].eid[j] = e;
                        } else if constexpr (VONLY) {
                            dst[j] = p.values + (size_t)e * L;
                        } else {
                            dst[5 * j] = p.values + (size_t)e * L;
                            dst[5 * j + 1] = p.grads + (size_t)e * 3 * L;
                            dst[5 * j + 2] = p.grads + (size_t)e * 3 * L + L;
                            dst[5 * j + 3] = p.grads + (size_t)e * 3 * L + 2 * L;
                            dst[5 * j + 4] = p.laps + (size_t)e * L;
                        }
                    }
                }
                if (ww == 0 && lane == 0) {
                    info[wi].cnt = cnt;
                    info[wi].n = N;
                }
                unsigned char *wdst = wbuf + wb * Cfg::W_BUF;
#pragma unroll
                for (int kx = 0; kx < 4; ++kx) {
                    const int c = 4 * kx + ww;
                    // the 4 weights (kz = 0..3) of each output, 0 past cnt
                    float w[NO][4];
#pragma unroll
                    for (int kz = 0; kz < 4; ++kz) {
                        if (j < cnt) {
                            const float X0 = X[kx][0], X1 = X[kx][1], X2 = X[kx][2];
                            const float Z0 = Z[kz][0], Z1 = Z[kz][1], Z2 = Z[kz][2];
                            w[0][kz] = nrm * (X0 * Y[0] * Z0);
                            if constexpr (!VONLY) {
                                const float gx = X1 * Y[0] * Z0, gy = X0 * Y[1] * Z0,
                                            gz = X0 * Y[0] * Z1;
                                w[1 % NO][kz] = nrm * (J[0] * gx + J[3] * gy + J[6] * gz);
                                w[2 % NO][kz] = nrm * (J[1] * gx + J[4] * gy + J[7] * gz);
                                w[3 % NO][kz] = nrm * (J[2] * gx + J[5] * gy + J[8] * gz);
                                const float hxx = X2 * Y[0] * Z0, hyy = X0 * Y[2] * Z0,
                                            hzz = X0 * Y[0] * Z2;
                                const float hxy = X1 * Y[1] * Z0, hxz = X1 * Y[0] * Z1,
                                            hyz = X0 * Y[1] * Z1;
                                w[4 % NO][kz] = nrm * (M[0] * hxx + M[1] * hyy + M[2] * hzz +
                                                       2.0f * (M[3] * hxy + M[4] * hxz + M[5] * hyz));
                            }
                        } else {
#pragma unroll
                            for (int o = 0; o < NO; ++o) w[o][kz] = 0.0f;
                        }
                    }
#pragma unroll
                    for (int o = 0; o < NO; ++o) {
                        const int r = NO * j + o;
                        if (r < N) {
                            // split into 16-bit planes; the 4 weights sit at
                            // window rows cz .. cz + 3 of the 8-row chunk
                            float rem[4] = {w[o][0], w[o][1], w[o][2], w[o][3]};
#pragma unroll
                            for (int pl = 0; pl < WPL; ++pl) {
                                uint64_t v64 = 0;
#pragma unroll
                                for (int kz = 0; kz < 4; ++kz) {
                                    const unsigned short bb = to_bits<T>(rem[kz]);
                                    rem[kz] -= from_bits<T>(bb);
                                    v64 |= (uint64_t)bb << (16 * kz);
                                }
                                const int sh = 16 * cz;
                                const uint64_t lo = cz == 4 ? 0ull : v64 << sh;
                                const uint64_t hi = cz == 0 ? 0ull : cz == 4 ? v64 : v64 >> (64 - sh);
                                uint4 v;
                                v.x = (uint32_t)lo;
                                v.y = (uint32_t)(lo >> 32);
                                v.z = (uint32_t)hi;
                                v.w = (uint32_t)(hi >> 32);
                                *reinterpret_cast<uint4 *>(wdst + (uint32_t)c * Cfg::KGROUP +
                                                           (uint32_t)(r + pl * Cfg::RLO) * 16u) = v;
                            }
                        }
                    }
                }
                // the tensor cores read the buffer through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                named_sync(1, 128);
                if (ww == 0 && lane == 0) mbar_arrive(w_full + wi);
                ++part;
            }
        }
        // no more parts
        if (ok && claim()) {
            if (ww == 0 && lane == 0) {
                info[part & 1].cnt = -1;
                mbar_arrive(w_full + (int)(part & 1));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

template <typename T, int APL, int MODE>
cudaError_t launch_tc_t(const EvalParams &p, const TcArgs &a, const CUtensorMap &tm,
                        const CUtensorMap &tm5, int sm_count, cudaStream_t stream)
{
    constexpr size_t smem = tc_smem<APL, MODE == 1>();
    static_assert(smem <= 227 * 1024, "stages and weight buffers exceed shared memory");
    static bool attr_set = false;   // raise this instantiation's dynamic shared-memory cap once
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(blip_eval_tc<T, APL, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int grid = std::max(1, std::min(sm_count, a.ncols));
    // the column counter of the CTAs' work queue starts at 0
    cudaError_t e = cudaMemsetAsync(a.col_ctr, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    blip_eval_tc<T, APL, MODE><<<grid, kThreads, smem, stream>>>(p, a, tm, tm5);
    return cudaGetLastError();
}

template <typename T, int APL>
cudaError_t launch_tc_v(const EvalParams &p, const TcArgs &a, const CUtensorMap &tm,
                        const CUtensorMap &tm5, int sm_count, cudaStream_t stream)
{
    if (a.ratio) return launch_tc_t<T, APL, 2>(p, a, tm, tm5, sm_count, stream);
    return p.grads == nullptr ? launch_tc_t<T, APL, 1>(p, a, tm, tm5, sm_count, stream)
                              : launch_tc_t<T, APL, 0>(p, a, tm, tm5, sm_count, stream);
}

PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn()
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

// Power-of-two scale of each component: the smallest 2^k >= max |a| (1 for
// an all-zero component), from the max |a| bits of the FP32 table.
__global__ void pow2_scales_kernel(const unsigned int *bits, int n, float *scales)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const float m = __uint_as_float(bits[l]);
    int e = 0;
    const float f = frexpf(m, &e);                      // m = f 2^e, f in [0.5, 1)
    scales[l] = m > 0.0f ? ldexpf(1.0f, f == 0.5f ? e - 1 : e) : 1.0f;
}

// hi, lo FP16 planes [2][n] of an FP32 table (rows of row_stride
// components): v = a / s_l (exact), hi = RN(v), lo = RN(v - hi).
__global__ void split_pairs_kernel(const float *src, long long n, long long row_stride,
                                   const float *scales, __half *dst)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v = src[i] / scales[i % row_stride];
        const __half h = __float2half_rn(v);
        dst[i] = h;
        dst[n + i] = __float2half_rn(v - __half2float(h));
    }
}

}  // namespace

cudaError_t make_tc_tmap(const void *base, int elem, long long row_stride, long long rows_total,
                         TmaDesc *out)
{
    if (!out || row_stride < kMT || rows_total < 1 || (elem != ELEM_BF16 && elem != ELEM_F16))
        return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const CUtensorMapDataType dt =
        elem == ELEM_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[2] = {(cuuint64_t)row_stride, (cuuint64_t)rows_total};
    const cuuint64_t strides[1] = {(cuuint64_t)row_stride * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)kWin};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap *>(out), dt, 2, const_cast<void *>(base), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_tc_tmap5(const void *base, int elem, long long row_stride, int n12, int n3,
                          int planes, long long plane_rows, int box_slabs, TmaDesc *out)
{
    if (box_slabs != 1 && box_slabs != 2) return cudaErrorInvalidValue;
    if (!out || row_stride < kMT || row_stride % 64 || (elem != ELEM_BF16 && elem != ELEM_F16) ||
        planes < 1 || planes > 2)
        return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const CUtensorMapDataType dt =
        elem == ELEM_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t row_bytes = (cuuint64_t)row_stride * 2;
    // components within a 64-component slab, rows of a grid column, grid
    // columns, slabs, planes
    const cuuint64_t dims[5] = {64, (cuuint64_t)(n3 + 3), (cuuint64_t)n12,
                                (cuuint64_t)(row_stride / 64), (cuuint64_t)planes};
    const cuuint64_t strides[4] = {row_bytes, row_bytes * (cuuint64_t)(n3 + 3), 128,
                                   row_bytes * (cuuint64_t)plane_rows};
    const cuuint32_t box[5] = {64, (cuuint32_t)kWin, 4, (cuuint32_t)box_slabs, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap *>(out), dt, 5, const_cast<void *>(base), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_split_pairs(const float *src, long long rows, long long row_stride, int Lreal,
                              unsigned int *bits, float *scales, void *dst, cudaStream_t stream)
{
    // padding components past Lreal are zero: their scale is 1
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned int) * (size_t)row_stride, stream);
    if (e == cudaSuccess) e = launch_absmax(src, rows, row_stride, Lreal, bits, stream);
    if (e == cudaSuccess) {
        pow2_scales_kernel<<<(unsigned)((row_stride + 255) / 256), 256, 0, stream>>>(
            bits, (int)row_stride, scales);
        e = cudaGetLastError();
    }
    const long long n = rows * row_stride;
    if (e == cudaSuccess) {
        const long long blocks = std::min<long long>((n + 255) / 256, 65535LL * 8);
        split_pairs_kernel<<<(unsigned)std::max<long long>(1, blocks), 256, 0, stream>>>(
            src, n, row_stride, scales, static_cast<__half *>(dst));
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_tc(const EvalParams &p, int elem, const int *cell_end, const int *cols,
                      int ncols, long long plane_rows, const TmaDesc &tmap, const TmaDesc *tmap5,
                      int *col_ctr, int sm_count, int stall, cudaStream_t stream,
                      const float *rcols, float *ratio)
{
    if (!p.perm || !cell_end || !cols || !col_ctr || ncols < 1 || p.n_k || plane_rows >= (1LL << 31) ||
        (ratio != nullptr) != (rcols != nullptr) || (ratio && p.grads))
        return cudaErrorInvalidValue;
    TcArgs a{};
    a.cell_end = cell_end;
    a.cols = cols;
    a.ncols = ncols;
    a.P = (int)sort_key_count(p.geo);
    a.mt = (p.Lreal + kMT - 1) / kMT;
    a.plane_rows = (int)plane_rows;
    a.stall = stall;
    a.wide = tmap5 != nullptr;
    a.col_ctr = col_ctr;
    a.rcols = rcols;
    a.ratio = ratio;
    const CUtensorMap &tm = *reinterpret_cast<const CUtensorMap *>(&tmap);
    const CUtensorMap &tm5 = *reinterpret_cast<const CUtensorMap *>(tmap5 ? tmap5 : &tmap);
    switch (elem) {
    case ELEM_F32: return launch_tc_v<__half, 2>(p, a, tm, tm5, sm_count, stream);
    case ELEM_BF16: return launch_tc_v<__nv_bfloat16, 1>(p, a, tm, tm5, sm_count, stream);
    case ELEM_F16: return launch_tc_v<__half, 1>(p, a, tm, tm5, sm_count, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace blip

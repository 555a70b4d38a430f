// Tensor-core kernel for the fused quasi-simultaneous ratio of dense sorted
// batches, with the inverse Slater columns as the second operand.
//
// For the trial move r'_j of electron j the ratio and its derivatives are
// (Sec. IV.A, Eq. 11.12.23.1 with the orbitals of Eq. 11.12.24.1)
//     R_o(j) = sum_l psi_{o,l}(r'_j) c_j[l]
//            = sum_k W_o^{(j)}[k] sum_l a[k][l] c_j[l],
// c_j the column (D^{-1})_{. j}, a[k][l] the coefficients of stencil row k,
// W_o^{(j)} the electron's five weights (value, gradient, Laplacian) on its
// 64 sites.  The orbital sum runs first, on the tensor cores, for a part of
// up to 25 electrons of at most 5 cells of one grid column (the parts of the
// evaluation kernel, whose stencils lie in 128 union rows k):
//     Y[k][j] = sum_l a[k][l] c'_j[l]     M = 128 union rows, K = orbitals,
//                                         N = the part's electrons,
// accumulated in FP32 in tensor memory over the part's orbital tiles; the
// epilogue then forms each electron's weights on the lane of its union row
// and reduces sum_k W_o^{(j)}[k] Y[k][j] over the 128 rows (a butterfly over
// the lanes, then the four lane quarters in a fixed order).  Against the
// ratio epilogue of the evaluation kernel, the per-column work of the
// epilogue (128 columns per orbital tile) becomes per-part work (5 numbers
// per electron), and the new orbital row is not formed: this kernel serves
// calls without it.
//
// Operands: the table tiles of the evaluation kernel in the K-major layout
// (8-row, 128-byte-swizzled atoms of stencil column c at c KB, the second
// 64-component half 16 KB on); c'_j[l] = c_j[l] s_l / sigma_j (s_l the table
// component's scale, sigma_j a power of two at or above max_l |c_j[l] s_l|
// for FP16 operands, from a pre-pass over the columns; 1 for BF16) split
// into two 16-bit parts (hi + lo) stacked along N (rows 0..31 hi, 32..63
// lo), built on the chip per orbital tile into a 4-slot ring by 8 warps
// from the columns in global memory (asked into L2 one part ahead).  One
// bulk copy per electron and tile would be the obvious staging, but the copy
// engine then issues ~30 small copies per tile and binds the kernel.  FP32 tables enter as their two scaled FP16
// planes: hi plane x (hi + lo), lo plane x hi.
//
// Persistent grid, one CTA per SM, 14 warps, the columns from the shared
// work queue of the evaluation kernel:
//   warp 0      takes columns, passes them on through a 4-slot ring; TMA
//               producer of the table tiles (4-stage ring);
//   warp 1      tensor memory and the MMAs (one thread): per part and
//               orbital tile, 8 K steps x planes into the part's 64-column
//               accumulator (one of four);
//   warps 2-5   epilogue, one per lane quarter: Y from tensor memory, the
//               weights of the lane's union row, the reductions;
//   warps 6-13  the part's electron geometry (with its 1-D B-spline factors
//               for the epilogue) and the c' tiles (two K groups of 8
//               orbitals per warp, lane = electron).
// Every wait is bounded (about 2 s); on a timeout every role winds down as in
// the evaluation kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "blip_tc_common.cuh"

namespace blip {

namespace {

constexpr int kRStages = 4;                     // table tile stages (32 KB)
constexpr int kRBSlots = 4;                     // c' tile slots
constexpr uint32_t kRKG = 64 * 16;              // one K group of a c' tile: 64 rows x 16 B
constexpr uint32_t kRB = 16 * kRKG;             // one c' tile: 128 orbitals (16 KB)
constexpr int kRAcc = 4;                        // accumulators
constexpr int kRAccCols = 64;                   // hi and lo c' columns of 32 electrons
constexpr uint32_t kRTmemCols = 256;
constexpr int kREpi = 4;                        // epilogue warps (one per lane quarter)
constexpr int kRC = 8;                          // operand warps (2 K groups of a tile each)
static_assert(2 + kREpi + kRC == kThreads / 32, "the ratio kernel's roles fill the block");

struct __align__(16) RPart {
    int cnt;            // electrons, or -1 for "no more parts"
    int pad[3];
    int cz[32];         // electron j: window row of its first stencil row
    int eid[32];        // electron index
    float sig[32];      // sigma_j
    float fac[32][36];  // electron j: 1-D factors [axis][site k][value, d1, d2]
};

constexpr size_t ratio_tc_smem()
{
    return kRStages * kStage + kRBSlots * kRB + 2 * sizeof(RPart) +
           2 * 4 * 32 * 5 * sizeof(float) + 512;
}

template <typename T, int APL>
__global__ void __launch_bounds__(kThreads, 1)
    blip_ratio_tc(EvalParams p, TcArgs a, const __grid_constant__ CUtensorMap tmap,
                  const __grid_constant__ CUtensorMap tmap5k)
{
    constexpr int FMT = std::is_same<T, __nv_bfloat16>::value ? 1 : 0;
    constexpr bool SIG = !std::is_same<T, __nv_bfloat16>::value;   // FP16 operands are scaled
    extern __shared__ __align__(1024) unsigned char smem[];
    if (smem_addr(smem) & 1023u) {
        if (threadIdx.x == 0) atomicOr(p.status, BLIP_STATUS_LAYOUT);
        return;
    }
    unsigned char *stageA = smem;
    unsigned char *bring = smem + kRStages * kStage;
    RPart *info = reinterpret_cast<RPart *>(bring + kRBSlots * kRB);
    float *qsum = reinterpret_cast<float *>(info + 2);          // [2][4 quarters][32][5]
    uint64_t *bars = reinterpret_cast<uint64_t *>(qsum + 2 * 4 * 32 * 5);
    uint64_t *a_full = bars, *a_empty = a_full + kRStages;
    uint64_t *b_full = a_empty + kRStages, *b_empty = b_full + kRBSlots;
    uint64_t *w_full = b_empty + kRBSlots, *w_empty = w_full + 2, *epi_done = w_empty + 2;
    uint64_t *acc_full = epi_done + 2, *acc_empty = acc_full + kRAcc;
    uint64_t *red_done = acc_empty + kRAcc, *drain = red_done + 2;
    uint64_t *cq_full = drain + 1, *cq_empty = cq_full + kColQ;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(cq_empty + kColQ);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *colq = abort_flag + 1;
    volatile int *decision = colq + kColQ;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n2 = p.geo.n[1], n3 = p.geo.n[2];
    check_offsets(p);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kRStages; ++s) {
            mbar_init(a_full + s, 1);
            mbar_init(a_empty + s, 1);
        }
        for (int s = 0; s < kRBSlots; ++s) {
            mbar_init(b_full + s, kRC);              // the operand warps
            mbar_init(b_empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(w_full + b, 1);
            mbar_init(w_empty + b, 1);
            mbar_init(epi_done + b, kREpi);
            mbar_init(red_done + b, 32 * kREpi);
        }
        for (int b = 0; b < kRAcc; ++b) {
            mbar_init(acc_full + b, 1);
            mbar_init(acc_empty + b, kREpi);
        }
        mbar_init(drain, 1);
        for (int q = 0; q < kColQ; ++q) {
            mbar_init(cq_full + q, 1);
            mbar_init(cq_empty + q, kRC);
        }


        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(kRTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- columns and TMA producer ----------------
        long long fill = 0;
        bool ok = true;
        // stage layout (K-major A): stencil column c = 4 kx + ky at c KB,
        // component half h at h 16 KB (one 128-byte-swizzled 8-row atom each)
        const int c = lane >> 1, h = lane & 1;       // narrow boxes: column c, half h
        const int kxl = c >> 2, kyl = c & 3;
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
                // empty columns are skipped: every pushed column has a part
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
            // memory unless they wrap around the cell: then one 4 KB box per
            // (kx, h) (5-D view), else 1 KB boxes
            const bool wide = a.wide && y >= 1 && y + 2 < n2;
            int gx = x - 1 + (wide ? (lane >> 1) : kxl), gy = y - 1 + kyl;
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
                for (int m = 0; m < a.mt && ok; ++m) {
                    for (int pl = 0; pl < APL; ++pl) {
                        const int s = (int)(fill % kRStages);
                        const long long k = fill / kRStages;
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
                            if (lane < 8)
                                tma_load_5d(st + (lane & 1) * 16384 + (lane >> 1) * 4096, &tmap5k, 0,
                                            z0, gx * n2 + y - 1, 2 * m + (lane & 1), pl, a_full + s);
                        } else {
                            tma_load_2d(st + h * 16384 + c * kBox, &tmap, m * kMT + 64 * h,
                                        pl * a.plane_rows + colrow + z0, a_full + s);
                        }
                        ++fill;
                    }
                }
            }
        }
        // drain: the copies of the last fills must land before the CTA exits
        for (long long f = fill > kRStages ? fill - kRStages : 0; f < fill; ++f) {
            const bool got = mbar_wait(a_full + (int)(f % kRStages), (unsigned)((f / kRStages) & 1));
            if (!__all_sync(FULL, got) && lane == 0) atomicOr(p.status, BLIP_STATUS_TIMEOUT);
        }


    } else if (warp == 1) {
        // ---------------- MMA issue (one thread) ----------------
        if (lane == 0) {
            bool ok = true, first = true;
            int s = 0, s_ph = 0, bs = 0, bs_ph = 0, ab = 0, ab_ph = 0, parts = 0;
            // K-major A: 8-row atoms 1 KB apart (SBO), the K offset inside the
            // 128-byte swizzle atom added to the start address; B: K groups
            // of 8 at kRKG bytes, N groups of 8 rows at 128 B
            const uint64_t a_desc0 = smem_desc(smem_addr(stageA), 16u, kBox, 2);
            const uint64_t b_desc0 = smem_desc(smem_addr(bring), kRKG, 128u, 0);
            const uint32_t id_both = instr_desc(kRAccCols, FMT, 0u);   // c' hi and lo
            const uint32_t id_hi = instr_desc(32, FMT, 0u);            // c' hi only
            for (int part = 0; ok; ++part) {
                const int wi = part & 1;
                if (!wait_bar(w_full + wi, (unsigned)((part >> 1) & 1), abort_flag)) {
                    raise_abort(p, abort_flag);
                    break;
                }
                if (info[wi].cnt < 0) break;
                if (parts >= kRAcc && !wait_bar(acc_empty + ab, (unsigned)(ab_ph ^ 1), abort_flag)) {
                    raise_abort(p, abort_flag);
                    break;
                }
                const uint32_t d = tmem + (uint32_t)(ab * kRAccCols);
                for (int m = 0; m < a.mt && ok; ++m) {
                    if (!wait_bar(b_full + bs, (unsigned)bs_ph, abort_flag)) {
                        raise_abort(p, abort_flag);
                        ok = false;
                        break;
                    }
                    const uint64_t bd0 = b_desc0 + (uint64_t)((bs * kRB) >> 4);
                    for (int pl = 0; pl < APL; ++pl) {
                        if (!wait_bar(a_full + s, (unsigned)s_ph, abort_flag)) {
                            raise_abort(p, abort_flag);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad0 = a_desc0 + (uint64_t)((s * kStage) >> 4);
                        // of an FP32 table's planes the lo one meets the hi
                        // part of c' only (lo x lo is below 2^-22 relative)
                        const uint32_t id = pl == 1 ? id_hi : id_both;
#pragma unroll
                        for (int ks = 0; ks < kMT / 16; ++ks) {
                            // orbitals 16 ks .. 16 ks + 15: half ks / 4, 32 bytes
                            // (ks % 4) into the swizzle atom; c' K groups 2 ks, 2 ks + 1
                            const uint64_t ad = ad0 + (uint64_t)(((ks >> 2) * 16384 + (ks & 3) * 32) >> 4);
                            const uint64_t bd = bd0 + (uint64_t)((ks * 2 * kRKG) >> 4);
                            mma_f16(d, ad, bd, id, (m == 0 && pl == 0 && ks == 0) ? 0u : 1u);
                        }
                        if (!(a.stall && first)) mma_commit(a_empty + s);
                        first = false;
                        if (++s == kRStages) {
                            s = 0;
                            s_ph ^= 1;
                        }
                    }
                    if (!ok) break;
                    mma_commit(b_empty + bs);
                    if (++bs == kRBSlots) {
                        bs = 0;
                        bs_ph ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(acc_full + ab);
                mma_commit(w_empty + wi);
                ++parts;
                if (++ab == kRAcc) {
                    ab = 0;
                    ab_ph ^= 1;
                }
            }
            mma_commit(drain);
            if (!mbar_wait(drain, 0)) atomicOr(p.status, BLIP_STATUS_TIMEOUT);
        }
        __syncwarp();
    } else if (warp < 2 + kREpi) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;
        const int et = threadIdx.x - 64;
        // positions without a cell (last sort bucket): NaN ratios
        {
            const int nan0 = a.cell_end[a.P - 1];
            for (int sl = nan0; sl < p.n_elec; ++sl) {
                if ((sl - nan0) % (int)gridDim.x != (int)blockIdx.x) continue;
                const size_t e = (size_t)p.perm[sl];
                if (et == 0) {
                    int bad = BLIP_STATUS_NONFINITE_POS;
                    if (p.georec) bad |= p.georec[sl].bad;
                    atomicOr(p.status, bad);
                }
                if (et < 5) a.ratio[e * 5 + et] = __int_as_float(0x7fc00000);
            }
        }
        // this lane's union row k = 32 q + lane: stencil column 4 kx + ky,
        // window row r
        const int k = 32 * q + lane;
        const int kx = k >> 5, ky = (k >> 3) & 3, r = k & 7;
        int ab = 0, ab_ph = 0;
        for (int part = 0;; ++part) {
            const int wi = part & 1;
            const unsigned ph = (unsigned)((part >> 1) & 1);
            if (!wait_bar(w_full + wi, ph, abort_flag)) {
                if (lane == 0) raise_abort(p, abort_flag);
                break;
            }
            const int cnt = info[wi].cnt;
            if (cnt < 0) break;
            if (!wait_bar(acc_full + ab, (unsigned)ab_ph, abort_flag)) {
                if (lane == 0) raise_abort(p, abort_flag);
                break;
            }
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * kRAccCols);
            float *qs = qsum + wi * (4 * 32 * 5) + q * (32 * 5);
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {   // electrons 16 half .. 16 half + 15
                uint32_t yh[16], yl[16];
                tmem_ld16_nowait(taddr + 16 * half, yh);
                tmem_ld16_nowait(taddr + 32 + 16 * half, yl);
                tmem_wait_ld();
                if (half == 1) {
                    // both halves are in registers: the accumulator is free
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acc_empty + ab);
                    if (++ab == kRAcc) {
                        ab = 0;
                        ab_ph ^= 1;
                    }
                }
                // two groups of 8 electrons: the weights of this row times Y,
                // then over the 32 lanes (lane L ends with electron L / 4 of the
                // group after the butterfly)
#pragma unroll
                for (int grp = 0; grp < 2; ++grp) {

                    float pv[5][8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = 16 * half + 8 * grp + u;
                        const float yv = __uint_as_float(yh[8 * grp + u]) + __uint_as_float(yl[8 * grp + u]);
                        float w[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                        if (j < cnt) {
                            const int kz = r - info[wi].cz[j];
                            if (kz >= 0 && kz <= 3) {
                                // the weights of site (kx, ky, kz), as site_weights forms them
                                const float *f = info[wi].fac[j];
                                const float X0 = f[3 * kx], X1 = f[3 * kx + 1], X2 = f[3 * kx + 2];
                                const float Y0 = f[12 + 3 * ky], Y1 = f[13 + 3 * ky], Y2 = f[14 + 3 * ky];
                                const float Z0 = f[24 + 3 * kz], Z1 = f[25 + 3 * kz], Z2 = f[26 + 3 * kz];
                                const float *J = p.geo.J, *M = p.geo.M;
                                const float nrm = p.geo.norm;
                                const float gx = X1 * Y0 * Z0, gy = X0 * Y1 * Z0, gz = X0 * Y0 * Z1;
                                const float hxx = X2 * Y0 * Z0, hyy = X0 * Y2 * Z0, hzz = X0 * Y0 * Z2;
                                const float hxy = X1 * Y1 * Z0, hxz = X1 * Y0 * Z1, hyz = X0 * Y1 * Z1;
                                w[0] = nrm * (X0 * Y0 * Z0);
                                w[1] = nrm * (J[0] * gx + J[3] * gy + J[6] * gz);
                                w[2] = nrm * (J[1] * gx + J[4] * gy + J[7] * gz);
                                w[3] = nrm * (J[2] * gx + J[5] * gy + J[8] * gz);
                                w[4] = nrm * (M[0] * hxx + M[1] * hyy + M[2] * hzz +
                                              2.0f * (M[3] * hxy + M[4] * hxz + M[5] * hyz));
                            }
                        }
#pragma unroll
                        for (int o = 0; o < 5; ++o) pv[o][u] = w[o] * yv;
                    }
#pragma unroll
                    for (int o = 0; o < 5; ++o) {
#pragma unroll
                        for (int st = 0; st < 3; ++st) {
                            const int off = 16 >> st, hh = 4 >> st;
                            const bool up = (lane & off) != 0;
#pragma unroll
                            for (int i = 0; i < hh; ++i) {
                                const float send = up ? pv[o][i] : pv[o][i + hh];
                                const float keep = up ? pv[o][i + hh] : pv[o][i];
                                pv[o][i] = keep + __shfl_xor_sync(FULL, send, off);
                            }
                        }
                        pv[o][0] += __shfl_xor_sync(FULL, pv[o][0], 2);
                        pv[o][0] += __shfl_xor_sync(FULL, pv[o][0], 1);
                    }
                    if ((lane & 3) == 0) {
                        const int j = 16 * half + 8 * grp + (lane >> 2);
#pragma unroll
                        for (int o = 0; o < 5; ++o) qs[j * 5 + o] = pv[o][0];
                    }
                }
            }
            mbar_arrive(red_done + wi);                  // all 32 kREpi threads
            if (!wait_bar(red_done + wi, ph, abort_flag)) {
                if (lane == 0) raise_abort(p, abort_flag);
                break;
            }
            if (et < 5 * cnt) {
                const float *q0 = qsum + wi * (4 * 32 * 5);
                const float tot = ((q0[et] + q0[160 + et]) + q0[320 + et]) + q0[480 + et];
                const int j = et / 5;
                a.ratio[(size_t)info[wi].eid[j] * 5 + et % 5] = tot * info[wi].sig[j];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(epi_done + wi);
        }
    } else {
        // ---------------- electron geometry and c' tiles ----------------
        const int ww = warp - 2 - kREpi;
        const size_t L = (size_t)p.Lreal;
        // 16-byte loads of the columns when every row starts 16-byte aligned
        const bool vec = (p.Lreal & 3) == 0 && (reinterpret_cast<uintptr_t>(a.rcols) & 15u) == 0;
        bool ok = true;
        int part = 0, bs = 0, bs_ph = 0, built = 0;
        auto claim = [&]() -> bool {
            const int wi = part & 1;
            bool got = true;
            if (part >= 2) {
                const unsigned ph = (unsigned)(((part >> 1) - 1) & 1);
                got = wait_bar(w_empty + wi, ph, abort_flag);
                if (got) got = wait_bar(epi_done + wi, ph, abort_flag);
            }
            if (!__all_sync(FULL, got) && lane == 0) raise_abort(p, abort_flag);
            // one thread reads the abort flag between two barriers, so the four
            // warps take the same decision (and meet the same barriers after it)
            named_sync(1, 32 * kRC);
            if (ww == 0 && lane == 0) *decision = *abort_flag;
            named_sync(1, 32 * kRC);
            return !*decision;
        };
        int taken = 0;
        auto take = [&]() -> int {
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
        // one part ahead: the next part's electrons are found, and their
        // columns asked into L2, while this part's tiles are built, so the
        // producer's bulk copies of them hit L2 (warp ww: a quarter of the
        // 128-byte lines of each column)
        int nz0 = 0, ns0 = 0, ncnt = 0, ne = 0;
        auto look_ahead = [&]() -> bool {
            if (!advance(nz0, ns0, ncnt)) return false;
            ne = lane < ncnt ? p.perm[ns0 + lane] : 0;
            if (lane < ncnt) {
                const float *row = a.rcols + (size_t)ne * L;
                for (int l = 32 * ww; l < p.Lreal; l += 32 * kRC)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(row + l));
            }
            return true;
        };
        bool have = look_ahead();
        while (ok && have) {
            const int z0 = nz0, s0 = ns0, cnt = ncnt;
            const int e_next = ne;
            have = look_ahead();
            if (!claim()) {
                ok = false;
                break;
            }
            const int wi = part & 1;
            const int j = lane;
            int e = 0;
            if (j < cnt) {
                const int slot = s0 + j;
                e = e_next;
                int i2, bad;
                float t0, t1, t2;
                if (p.georec) {
                    const ElecGeo g = p.georec[slot];
                    i2 = g.i[2];
                    bad = g.bad;
                    t0 = g.t[0];
                    t1 = g.t[1];
                    t2 = g.t[2];
                } else {
                    const double *rp = p.pos + 3 * (size_t)e;
                    int i0, i1;
                    bad = wrap_axis(p.geo, 0, rp[0], rp[1], rp[2], i0, t0);
                    bad |= wrap_axis(p.geo, 1, rp[0], rp[1], rp[2], i1, t1);
                    bad |= wrap_axis(p.geo, 2, rp[0], rp[1], rp[2], i2, t2);
                }
                // the sort put the electron in one of the part's cells; clamp
                // anyway so that its rows stay inside the 8-row window
                const int cz = min(max(i2 - z0, 0), kSegCells - 1);
                if (ww == 0) {
                    if (bad) atomicOr(p.status, bad);
                    info[wi].cz[j] = cz;
                    info[wi].eid[j] = e;
                }
                // the 1-D factors of axis ww for the epilogue (no lane-dependent
                // site index there, so no divergent branches)
                if (ww < 3) {
                    const float ta = ww == 0 ? t0 : ww == 1 ? t1 : t2;
                    float *f = &info[wi].fac[j][12 * ww];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) bspline_1d(ta, kk, f[3 * kk], f[3 * kk + 1], f[3 * kk + 2]);
                }
            }
            const float *crow = a.rcols + (size_t)e * L;
            // sigma_j (FP16 operands): a power of two at or above
            // max_l |c_j[l] s_l|, from the pre-pass over the columns
            const float sig = (SIG && j < cnt) ? a.rsig[e] : 1.0f;
            if (ww == 0 && j < cnt) info[wi].sig[j] = sig;
            const float rsig = 1.0f / sig;                   // a power of two: exact
            if (ww == 0 && lane == 0) info[wi].cnt = cnt;
            __syncwarp();
            named_sync(1, 32 * kRC);
            if (ww == 0 && lane == 0) mbar_arrive(w_full + wi);
            // c' tiles: warp ww the K groups 4 ww .. 4 ww + 3 (orbitals
            // 32 ww .. 32 ww + 31 of the tile); row j hi, row 32 + j lo
            for (int m = 0; m < a.mt && ok; ++m) {
                if (built >= kRBSlots &&
                    !__all_sync(FULL, wait_bar(b_empty + bs, (unsigned)(bs_ph ^ 1), abort_flag))) {
                    if (lane == 0) raise_abort(p, abort_flag);
                    ok = false;
                    break;
                }
                unsigned char *tile = bring + bs * kRB;
                // the lane's 16 orbitals of the tile (K groups 2 ww, 2 ww + 1)
                // and their scales, all loads issued before any use (the
                // column segments were asked into L2 a part ahead)
                const int lb = m * kMT + 16 * ww;
                float v[16], sv[16];
                if (vec && lb + 16 <= p.Lreal) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 c4 = j < cnt ? __ldcs(reinterpret_cast<const float4 *>(crow + lb) + u)
                                                  : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        const float4 s4 = p.scales ? __ldg(reinterpret_cast<const float4 *>(p.scales + lb) + u)
                                                   : make_float4(1.0f, 1.0f, 1.0f, 1.0f);
                        v[4 * u] = c4.x; v[4 * u + 1] = c4.y; v[4 * u + 2] = c4.z; v[4 * u + 3] = c4.w;
                        sv[4 * u] = s4.x; sv[4 * u + 1] = s4.y; sv[4 * u + 2] = s4.z; sv[4 * u + 3] = s4.w;
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int l = lb + u;
                        v[u] = (j < cnt && l < p.Lreal) ? __ldcs(crow + l) : 0.0f;
                        sv[u] = (p.scales && l < p.Lreal) ? __ldg(p.scales + l) : 1.0f;
                    }
                }
#pragma unroll
                for (int gg = 0; gg < 2; ++gg) {
                    const int g = 2 * ww + gg;
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        float x0 = v[8 * gg + u] * sv[8 * gg + u];
                        float x1 = v[8 * gg + u + 1] * sv[8 * gg + u + 1];
                        if (SIG) {
                            x0 *= rsig;
                            x1 *= rsig;
                        }
                        // hi = RN(x), lo = RN(x - hi), two values per conversion
                        const uint32_t hp = pack2<T>(x0, x1);
                        const float2 hb = unpack2<T>(hp);
                        hw[u >> 1] = hp;
                        lw[u >> 1] = pack2<T>(x0 - hb.x, x1 - hb.y);
                    }
                    *reinterpret_cast<uint4 *>(tile + g * kRKG + j * 16) =
                        make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(tile + g * kRKG + (32 + j) * 16) =
                        make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
                // the tensor cores read the tile through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(b_full + bs);
                ++built;
                if (++bs == kRBSlots) {
                    bs = 0;
                    bs_ph ^= 1;
                }
            }
            ++part;
        }
        // no more parts
        if (ok && claim()) {
            if (ww == 0 && lane == 0) {
                info[part & 1].cnt = -1;
                mbar_arrive(w_full + (part & 1));
            }
        }

    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kRTmemCols)
                     : "memory");
    }
}

// sigma_e: the smallest power of two at or above max_l |c_e[l] s_l| (1 for
// a zero column); one warp per electron (vec: 16-byte loads).
__global__ void ratio_sigma_kernel(const float *__restrict__ cols, int n_elec, int L,
                                   const float *__restrict__ scales, int vec,
                                   float *__restrict__ sig)
{
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n_elec; e += nw) {
        const float *row = cols + e * (long long)L;
        float mx = 0.0f;
        if (vec) {
            for (int l = 4 * lane; l < L; l += 128) {
                const float4 c = __ldg(reinterpret_cast<const float4 *>(row + l));
                float4 s = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
                if (scales) s = __ldg(reinterpret_cast<const float4 *>(scales + l));
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(c.x * s.x), fabsf(c.y * s.y)),
                                     fmaxf(fabsf(c.z * s.z), fabsf(c.w * s.w))));
            }
        } else {
            for (int l = lane; l < L; l += 32)
                mx = fmaxf(mx, fabsf(__ldg(row + l) * (scales ? __ldg(scales + l) : 1.0f)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
        if (lane == 0) {
            float sg = 1.0f;
            if (mx > 0.0f) {
                int ex = 0;
                const float f = frexpf(mx, &ex);          // mx = f 2^ex, f in [0.5, 1)
                sg = ldexpf(1.0f, f == 0.5f ? ex - 1 : ex);
            }
            sig[e] = sg;
        }
    }
}

template <typename T, int APL>
cudaError_t launch_ratio_tc_t(const EvalParams &p, const TcArgs &a, const CUtensorMap &tm,
                              const CUtensorMap &tm5k, int sm_count, cudaStream_t stream)
{
    constexpr size_t smem = ratio_tc_smem();
    static_assert(smem <= 227 * 1024, "stages and tiles exceed shared memory");
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(blip_ratio_tc<T, APL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int grid = std::max(1, std::min(sm_count, a.ncols));
    cudaError_t e = cudaMemsetAsync(a.col_ctr, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    if (!std::is_same<T, __nv_bfloat16>::value) {
        const long long blocks = std::min<long long>(((long long)p.n_elec + 7) / 8, 65535LL * 16);
        ratio_sigma_kernel<<<(unsigned)std::max<long long>(1, blocks), 256, 0, stream>>>(
            a.rcols, p.n_elec, p.Lreal, p.scales,
            (p.Lreal % 4) == 0 && (reinterpret_cast<uintptr_t>(a.rcols) & 15u) == 0,
            const_cast<float *>(a.rsig));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    blip_ratio_tc<T, APL><<<grid, kThreads, smem, stream>>>(p, a, tm, tm5k);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ratio_tc(const EvalParams &p, int elem, const int *cell_end, const int *cols,
                            int ncols, long long plane_rows, const TmaDesc &tmap,
                            const TmaDesc *tmap5k, int *col_ctr, int sm_count, int stall,
                            cudaStream_t stream, const float *rcols, float *ratio, float *sig)
{
    if (!p.perm || !cell_end || !cols || !col_ctr || !rcols || !ratio || ncols < 1 || p.n_k ||
        p.values || p.grads || plane_rows >= (1LL << 31) || (!sig && elem != ELEM_BF16))
        return cudaErrorInvalidValue;
    TcArgs a{};
    a.cell_end = cell_end;
    a.cols = cols;
    a.ncols = ncols;
    a.P = (int)sort_key_count(p.geo);
    a.mt = (p.Lreal + kMT - 1) / kMT;
    a.plane_rows = (int)plane_rows;
    a.stall = stall;
    a.wide = tmap5k != nullptr;
    a.col_ctr = col_ctr;
    a.rcols = rcols;
    a.ratio = ratio;
    a.rsig = sig;
    const CUtensorMap &tm = *reinterpret_cast<const CUtensorMap *>(&tmap);
    const CUtensorMap &tm5k = *reinterpret_cast<const CUtensorMap *>(tmap5k ? tmap5k : &tmap);
    switch (elem) {
    case ELEM_F32: return launch_ratio_tc_t<__half, 2>(p, a, tm, tm5k, sm_count, stream);
    case ELEM_BF16: return launch_ratio_tc_t<__nv_bfloat16, 1>(p, a, tm, tm5k, sm_count, stream);
    case ELEM_F16: return launch_ratio_tc_t<__half, 1>(p, a, tm, tm5k, sm_count, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace blip

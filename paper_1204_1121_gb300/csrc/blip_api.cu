// C ABI of libblip (declared in include/blip.h): table lifetime, evaluation
// entry points, status word, kernel choice, autotuning and CUDA graphs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "blip_internal.h"
#include "../../include/blip.h"

using namespace blip;

namespace {

int g_last_cuda_error = 0;

struct KernelChoice {
    int variant, chunks, warps, sort;
};

}  // namespace

struct blip_table_s {
    int device = 0;
    int sm_count = 0;
    int grid[3] = {0, 0, 0};
    int n_orb = 0, storage = 0, norm = 0, is_complex = 0;
    int elem = ELEM_F32;
    int Lreal = 0;
    int nchunk = 0;
    long long row_stride = 0;
    long long rows = 0;
    void *d_table = nullptr;
    size_t table_bytes = 0;
    float *d_scales = nullptr;
    int *d_status = nullptr;
    Geometry geo{};
    KernelChoice choice{VAR_REGISTER, 1, 8, 0};
    bool auto_mode = false;
    std::map<int, KernelChoice> tuned;   // by tune_key (batch size class, values-only mode)
    cudaStream_t last_stream = nullptr;
    bool used = false;
    // host-buffer entry point staging
    cudaStream_t own_stream = nullptr;
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // spatial-sort scratch (grown outside stream capture)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // test hook: stall the bulk kernel's pipeline (bounded waits run out)
    int test_stall = 0;
    // tensor maps of the table for the staged-tile kernel (tile depth 2, 4)
    TmaDesc tmap[2] = {};
    bool tmap_ok[2] = {false, false};
    // tensor-core kernel: grid-column keys in sort order, BF16 planes of an
    // FP32 table, the tensor map of its operand (made on first use)
    int *d_cols = nullptr;
    int *d_tc_ctr = nullptr;        // tensor-core kernel: the CTAs' column counter
    float *d_rsig = nullptr;        // ratio kernel: per-electron column scales
    int rsig_n = 0;
    int ncols = 0;
    void *d_planes = nullptr;
    float *d_tc_scales = nullptr;
    TmaDesc tc_tmap = {};
    TmaDesc tc_tmap5 = {};
    TmaDesc tc_tmap5k = {};         // the same view with one slab per box (ratio kernel)
    bool tc_wide = false;
    bool tc_ready = false;
    // L2 residency: access-policy window over the table (bytes, 0 = off) and
    // whether this table set the context's persisting-L2 limit
    size_t l2_window = 0;
    float l2_hit_ratio = 1.0f;
    bool l2_limit_set = false;
    // Bloch k-points (complex tables)
    int n_k = 0;
    int koff[kMaxKpoints + 1] = {};
    double kfrac[kMaxKpoints][3] = {};
    float kcart[kMaxKpoints][3] = {};
};

struct blip_graph_s {
    blip_table_s *table = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Test hook (blip_test_fail_alloc): while >= 0, the number of library device
// allocations that still succeed before one fails.
std::atomic<int> g_alloc_fail_after{-1};

// Every device allocation of the library goes through here.
template <typename T>
cudaError_t dev_alloc(T **p, size_t bytes)
{
    int n = g_alloc_fail_after.load();
    while (n >= 0) {
        if (g_alloc_fail_after.compare_exchange_weak(n, n - 1)) {
            if (n == 0) {                  // the injected failure; the hook disarms
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    void *v = nullptr;
    const cudaError_t e = cudaMalloc(&v, bytes);
    *p = static_cast<T *>(v);
    return e;
}

int cuda_fail(cudaError_t e)
{
    g_last_cuda_error = (int)e;
    return e == cudaErrorMemoryAllocation ? BLIP_ERR_OOM : BLIP_ERR_CUDA;
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// A with the lattice vectors as columns: A[c][i] = lattice[3 i + c].
// Fills geo.ainv (row-major A^{-1}), J = diag(n) A^{-1}, M = J J^T.
int make_geometry(const int grid[3], const double lattice[9], int norm, Geometry &geo)
{
    double A[3][3];
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) A[c][i] = lattice[3 * i + c];
    // inverse by Gauss-Jordan elimination with partial pivoting
    double m[3][6];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 6; ++c) m[r][c] = c < 3 ? A[r][c] : (c - 3 == r ? 1.0 : 0.0);
    double scale = 0.0;
    for (int i = 0; i < 3; ++i) {
        double nn = 0.0;
        for (int c = 0; c < 3; ++c) nn += lattice[3 * i + c] * lattice[3 * i + c];
        scale = std::max(scale, sqrt(nn));
    }
    if (!(scale > 0.0) || !isfinite(scale)) return BLIP_ERR_SINGULAR_LATTICE;
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(m[r][col]) > fabs(m[piv][col])) piv = r;
        if (fabs(m[piv][col]) <= 1e-12 * scale) return BLIP_ERR_SINGULAR_LATTICE;
        if (piv != col)
            for (int c = 0; c < 6; ++c) std::swap(m[piv][c], m[col][c]);
        const double d = m[col][col];
        for (int c = 0; c < 6; ++c) m[col][c] /= d;
        for (int r = 0; r < 3; ++r) {
            if (r == col) continue;
            const double f = m[r][col];
            for (int c = 0; c < 6; ++c) m[r][c] -= f * m[col][c];
        }
    }
    double J[3][3];
    for (int a = 0; a < 3; ++a) {
        geo.n[a] = grid[a];
        for (int c = 0; c < 3; ++c) {
            geo.ainv[3 * a + c] = m[a][3 + c];
            J[a][c] = grid[a] * m[a][3 + c];
            geo.J[3 * a + c] = (float)J[a][c];
        }
    }
    auto dot = [&](int a, int b) { return J[a][0] * J[b][0] + J[a][1] * J[b][1] + J[a][2] * J[b][2]; };
    geo.M[0] = (float)dot(0, 0);
    geo.M[1] = (float)dot(1, 1);
    geo.M[2] = (float)dot(2, 2);
    geo.M[3] = (float)dot(0, 1);
    geo.M[4] = (float)dot(0, 2);
    geo.M[5] = (float)dot(1, 2);
    geo.norm = norm == BLIP_NORM_ALFE_GILLAN ? 3.375f : 1.0f;
    return BLIP_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

void copy_kpoints(const blip_table_s *t, EvalParams &p)
{
    p.n_k = t->n_k;
    memcpy(p.koff, t->koff, sizeof(p.koff));
    memcpy(p.kfrac, t->kfrac, sizeof(p.kfrac));
    memcpy(p.kcart, t->kcart, sizeof(p.kcart));
}

int size_class(int n_elec)
{
    int c = 0;
    while (n_elec > 1) { n_elec >>= 1; ++c; }
    return c;
}

// Key of the tuned choices: batch size class and output mode (values only or
// all five outputs), which load the kernels differently.
int tune_key(int n_elec, bool values_only) { return 2 * size_class(n_elec) + (values_only ? 1 : 0); }

KernelChoice pick(const blip_table_s *t, int n_elec, bool values_only)
{
    if (t->auto_mode) {
        auto it = t->tuned.find(tune_key(n_elec, values_only));
        if (it != t->tuned.end()) return it->second;
    }
    return t->choice;
}

int validate_eval(const blip_table_s *t, const double *pos, int n_elec, const int *offs,
                  int n_walkers, const void *values, const void *grads, const void *laps)
{
    if (!t || n_elec < 0) return BLIP_ERR_INVALID_ARG;
    if (n_elec > 0 && (!pos || !values)) return BLIP_ERR_INVALID_ARG;
    if ((grads == nullptr) != (laps == nullptr)) return BLIP_ERR_INVALID_ARG;
    if (offs && n_walkers < 1) return BLIP_ERR_INVALID_ARG;
    return BLIP_OK;
}

// Spatial sort of the batch into the table's scratch (grown outside stream
// capture); *perm receives the evaluation order.
int sorted_order(blip_table_s *t, const double *pos, int n_elec, cudaStream_t stream, int **perm,
                 const ElecGeo **georec = nullptr)
{
    // sort scratch, then (optionally) per-electron geometry records by
    // electron and by slot
    const size_t sort_b = (sort_scratch_bytes(n_elec, t->geo) + 255) & ~(size_t)255;
    const size_t rec_b = sizeof(ElecGeo) * (size_t)n_elec;
    const size_t need = sort_b + (georec ? 2 * rec_b : 0);
    if (t->scratch_bytes < need) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(stream, &cs));
        if (cs != cudaStreamCaptureStatusNone) return BLIP_ERR_INVALID_ARG;  // no growth in capture
        if (t->scratch) {
            CK(cudaDeviceSynchronize());   // earlier sorted evaluations may use it on any stream
            cudaFree(t->scratch);
        }
        t->scratch = nullptr;
        t->scratch_bytes = 0;
        CK(dev_alloc(&t->scratch, need));
        t->scratch_bytes = need;
    }
    if (georec) {
        ElecGeo *by_e = reinterpret_cast<ElecGeo *>(static_cast<char *>(t->scratch) + sort_b);
        ElecGeo *by_slot = by_e + n_elec;
        CK(launch_sort(t->geo, pos, n_elec, t->scratch, perm, stream, by_e, by_slot));
        *georec = by_slot;
    } else {
        CK(launch_sort(t->geo, pos, n_elec, t->scratch, perm, stream));
    }
    return BLIP_OK;
}

// The table's tensor map for the staged-tile kernel with tile depth tz
// (encoded once, on first use).
int staged_tmap(blip_table_s *t, int tz, const TmaDesc **out)
{
    const int i = tz == 2 ? 0 : 1;
    if (!t->tmap_ok[i]) {
        CK(make_staged_tmap(t->d_table, t->elem, t->row_stride, t->rows, tz, &t->tmap[i]));
        t->tmap_ok[i] = true;
    }
    *out = &t->tmap[i];
    return BLIP_OK;
}

// The bulk-copy, staged-tile, split-stencil, persistent and tensor-core
// kernels have no Bloch epilogue.
bool has_bloch_epilogue(const KernelChoice &kc)
{
    return kc.variant != VAR_BULK && kc.variant != VAR_STAGED && kc.variant != VAR_SPLIT &&
           kc.variant != VAR_REGISTER_PERSIST && kc.variant != VAR_TENSOR;
}

// What the tensor-core kernel needs beyond the table, made once (outside
// stream capture): the keys of the grid columns' first cells in sort order,
// for FP32 tables their two scaled FP16 planes, and the operand tensor map.
int tc_prepare(blip_table_s *t)
{
    if (t->tc_ready) return BLIP_OK;
    std::vector<int> keys;
    keys.reserve((size_t)t->grid[0] * t->grid[1]);
    for (int x = 0; x < t->grid[0]; ++x)
        for (int y = 0; y < t->grid[1]; ++y) keys.push_back(sort_cell_key(t->geo, x, y, 0));
    std::sort(keys.begin(), keys.end());
    if (!t->d_tc_ctr) CK(dev_alloc(&t->d_tc_ctr, sizeof(int)));
    if (!t->d_cols) {
        CK(dev_alloc(&t->d_cols, sizeof(int) * keys.size()));
        CK(cudaMemcpy(t->d_cols, keys.data(), sizeof(int) * keys.size(), cudaMemcpyHostToDevice));
        t->ncols = (int)keys.size();
    }
    const void *operand = t->d_table;
    long long rows_total = t->rows;
    if (t->elem == ELEM_F32) {
        if (2 * t->rows >= (1LL << 31)) return BLIP_ERR_INVALID_ARG;
        if (!t->d_planes) {
            const long long n = t->rows * t->row_stride;
            unsigned int *bits = nullptr;
            CK(dev_alloc(&t->d_tc_scales, sizeof(float) * (size_t)t->row_stride));
            CK(dev_alloc(&t->d_planes, (size_t)n * 2 * 2));
            CK(dev_alloc(&bits, sizeof(unsigned int) * (size_t)t->row_stride));
            cudaError_t e = launch_split_pairs(static_cast<const float *>(t->d_table), t->rows,
                                               t->row_stride, t->Lreal, bits, t->d_tc_scales,
                                               t->d_planes, t->own_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(t->own_stream);
            cudaFree(bits);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        operand = t->d_planes;
        rows_total = 2 * t->rows;
    }
    const int op_elem = t->elem == ELEM_F32 ? ELEM_F16 : t->elem;
    CK(make_tc_tmap(operand, op_elem, t->row_stride, rows_total, &t->tc_tmap));
    // the 5-D view for 8 KB boxes; without it the kernel uses 1 KB boxes only
    t->tc_wide = make_tc_tmap5(operand, op_elem, t->row_stride, t->grid[0] * t->grid[1],
                               t->grid[2], t->elem == ELEM_F32 ? 2 : 1, t->rows, 2,
                               &t->tc_tmap5) == cudaSuccess &&
                 make_tc_tmap5(operand, op_elem, t->row_stride, t->grid[0] * t->grid[1],
                               t->grid[2], t->elem == ELEM_F32 ? 2 : 1, t->rows, 1,
                               &t->tc_tmap5k) == cudaSuccess;
    t->tc_ready = true;
    return BLIP_OK;
}

// Launch parameters of an evaluation with kernel choice kc; the evaluation
// order (perm, georec) is left to the caller.
EvalParams make_params(const blip_table_s *t, const double *pos, int n_elec, const int *offs,
                       int n_walkers, void *values, void *grads, void *laps,
                       const KernelChoice &kc)
{
    EvalParams p{};
    p.table = t->d_table;
    p.scales = t->d_scales;
    p.row_stride = t->row_stride;
    p.Lreal = t->Lreal;
    p.nchunk = t->nchunk;
    const bool per_chunk = kc.variant == VAR_GROUPED || kc.variant == VAR_STAGED;
    p.groups = per_chunk ? t->nchunk : (t->nchunk + kc.chunks - 1) / kc.chunks;
    p.items = (long long)n_elec * p.groups;
    p.geo = t->geo;
    p.pos = pos;
    p.n_elec = n_elec;
    p.perm = nullptr;
    p.georec = nullptr;
    p.group_major = kc.sort == 2 ? 1 : 0;
    p.offsets = offs;
    p.n_walkers = offs ? n_walkers : 0;
    p.values = static_cast<float *>(values);
    p.grads = static_cast<float *>(grads);
    p.laps = static_cast<float *>(laps);
    p.vec_out = (t->Lreal % 4 == 0) && aligned16(values) &&
                (!grads || (aligned16(grads) && aligned16(laps)));
    p.status = t->d_status;
    copy_kpoints(t, p);
    return p;
}

// While alive, launches on stream carry the table's L2 access-policy window
// (hits persist, misses stream); the stream's previous window comes back
// afterwards.  Streams that take no window (the legacy default stream) are
// launched without it.
struct L2Window {
    cudaStream_t s = nullptr;
    cudaStreamAttrValue old{};
    bool set = false;
    L2Window(const blip_table_s *t, cudaStream_t stream) : s(stream)
    {
        if (!t->l2_window || !stream) return;
        if (cudaStreamGetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &old) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        cudaStreamAttrValue v{};
        v.accessPolicyWindow.base_ptr = t->d_table;
        v.accessPolicyWindow.num_bytes = t->l2_window;
        v.accessPolicyWindow.hitRatio = t->l2_hit_ratio;
        v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        set = cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &v) == cudaSuccess;
        if (!set) cudaGetLastError();
    }
    ~L2Window()
    {
        if (set && cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &old) != cudaSuccess)
            cudaGetLastError();
    }
};

// Launch kernel choice kc on prepared parameters; scratch holds the sort
// whose views the grouped and staged kernels read.
int launch_choice(blip_table_s *t, const EvalParams &p, const KernelChoice &kc, void *scratch,
                  cudaStream_t stream)
{
    if (t->n_k && !has_bloch_epilogue(kc)) return BLIP_ERR_INVALID_ARG;
    const L2Window window(t, stream);
    if (kc.variant == VAR_BULK) {
        const size_t smem = bulk_smem_bytes(kc.chunks, kc.warps);
        int per_sm = (int)((228 * 1024) / (smem + 1024));
        per_sm = std::max(1, std::min(per_sm, 4));
        CK(launch_bulk(p, t->elem, kc.chunks, kc.warps, per_sm, t->sm_count, t->test_stall,
                       stream));
    } else if (kc.variant == VAR_GROUPED) {
        const int *keys = nullptr, *cell_end = nullptr;
        sort_views(t->geo, p.n_elec, scratch, &keys, &cell_end);
        CK(launch_grouped(p, t->elem, kc.chunks, kc.warps, keys, cell_end, stream));
    } else if (kc.variant == VAR_STAGED) {
        const int *keys = nullptr, *cell_end = nullptr;
        sort_views(t->geo, p.n_elec, scratch, &keys, &cell_end);
        const TmaDesc *tm = nullptr;
        int rc = staged_tmap(t, kc.chunks, &tm);
        if (rc) return rc;
        CK(launch_staged(p, t->elem, kc.chunks, kc.warps, cell_end, *tm, t->sm_count, t->test_stall,
                         stream));
    } else if (kc.variant == VAR_TENSOR) {
        if (!t->tc_ready) return BLIP_ERR_INVALID_ARG;   // prepared by blip_set_kernel / autotune
        const int *keys = nullptr, *cell_end = nullptr;
        sort_views(t->geo, p.n_elec, scratch, &keys, &cell_end);
        EvalParams pt = p;
        if (t->elem == ELEM_F32) pt.scales = t->d_tc_scales;   // the planes' power-of-two scales
        CK(launch_tc(pt, t->elem, cell_end, t->d_cols, t->ncols, t->rows, t->tc_tmap,
                     t->tc_wide ? &t->tc_tmap5 : nullptr, t->d_tc_ctr, t->sm_count,
                     t->test_stall, stream));
    } else if (kc.variant == VAR_SPLIT) {
        CK(launch_split(p, t->elem, stream));
    } else if (kc.variant == VAR_REGISTER_PERSIST) {
        if (t->elem != ELEM_F32) return BLIP_ERR_INVALID_ARG;
        CK(launch_persist(p, kc.warps, t->sm_count, stream));
    } else {
        CK(launch_eval(p, t->elem, kc.variant, kc.chunks, kc.warps, stream));
    }
    t->last_stream = stream;
    t->used = true;
    return BLIP_OK;
}

int eval_device(blip_table_s *t, const double *pos, int n_elec, const int *offs, int n_walkers,
                void *values, void *grads, void *laps, cudaStream_t stream, const KernelChoice &kc)
{
    if (n_elec == 0) return BLIP_OK;
    if (t->n_k && !has_bloch_epilogue(kc)) return BLIP_ERR_INVALID_ARG;
    EvalParams p = make_params(t, pos, n_elec, offs, n_walkers, values, grads, laps, kc);
    if (kc.sort || kc.variant == VAR_GROUPED || kc.variant == VAR_STAGED ||
        kc.variant == VAR_TENSOR) {
        int *perm = nullptr;
        const ElecGeo *rec = nullptr;
        const bool want_rec = t->n_k == 0 && kc.variant != VAR_BULK;
        int rc = sorted_order(t, pos, n_elec, stream, &perm, want_rec ? &rec : nullptr);
        if (rc) return rc;
        p.perm = perm;
        p.georec = rec;
    }
    return launch_choice(t, p, kc, t->scratch, stream);
}

int grow_stage(blip_table_s *t, size_t bytes)
{
    if (t->stage_bytes >= bytes) return BLIP_OK;
    if (t->stage) cudaFree(t->stage);
    t->stage = nullptr;
    t->stage_bytes = 0;
    CK(dev_alloc(&t->stage, bytes));
    t->stage_bytes = bytes;
    return BLIP_OK;
}

void free_table(blip_table_s *t)
{
    if (!t) return;
    if (!t->d_table && !t->d_scales && !t->d_status && !t->stage && !t->scratch &&
        !t->own_stream && !t->d_cols && !t->d_planes && !t->d_tc_scales &&
        !t->d_tc_ctr && !t->d_rsig) {
        delete t;
        return;
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != t->device) cudaSetDevice(t->device);
    if (t->l2_limit_set) {
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0);
    }
    if (t->d_table) cudaFree(t->d_table);
    if (t->d_scales) cudaFree(t->d_scales);
    if (t->d_status) cudaFree(t->d_status);
    if (t->stage) cudaFree(t->stage);
    if (t->scratch) cudaFree(t->scratch);
    if (t->d_cols) cudaFree(t->d_cols);
    if (t->d_tc_ctr) cudaFree(t->d_tc_ctr);
    if (t->d_rsig) cudaFree(t->d_rsig);
    if (t->d_planes) cudaFree(t->d_planes);
    if (t->d_tc_scales) cudaFree(t->d_tc_scales);
    if (t->own_stream) cudaStreamDestroy(t->own_stream);
    if (cur >= 0 && cur != t->device) cudaSetDevice(cur);
    delete t;
}

int create_impl(const int grid[3], const double lattice[9], int n_orb, int storage, int norm,
                const void *coeffs, int coeffs_is_double, int coeffs_on_device, blip_table_s *t)
{
    int rc = make_geometry(grid, lattice, norm, t->geo);   // host-only checks first
    if (rc) return rc;
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return BLIP_ERR_NO_DEVICE;
    }
    CK(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3) return BLIP_ERR_NO_DEVICE;   // sm_103 only
    t->device = dev;
    t->sm_count = prop.multiProcessorCount;
    memcpy(t->grid, grid, sizeof(t->grid));
    t->n_orb = n_orb;
    t->storage = storage;
    t->norm = norm;
    t->is_complex = storage == BLIP_C64 || storage == BLIP_BF16PAIR;
    t->elem = (storage == BLIP_BF16 || storage == BLIP_BF16PAIR) ? ELEM_BF16
            : storage == BLIP_F16 ? ELEM_F16 : ELEM_F32;
    t->Lreal = n_orb * (t->is_complex ? 2 : 1);
    const int vec = elem_vec(t->elem);
    t->nchunk = (t->Lreal + 32 * vec - 1) / (32 * vec);
    t->row_stride = (long long)t->nchunk * 32 * vec;
    t->rows = (long long)grid[0] * grid[1] * (grid[2] + 3);
    const long long src_rows = (long long)grid[0] * grid[1] * grid[2];
    t->choice = KernelChoice{VAR_REGISTER, 1, 8, 0};

    CK(cudaStreamCreateWithFlags(&t->own_stream, cudaStreamNonBlocking));
    cudaStream_t s = t->own_stream;
    // A device source may still be being written by work the caller queued on
    // any stream (the library's stream does not order after the legacy
    // default stream): wait for the whole device before reading it.
    if (coeffs_on_device) CK(cudaDeviceSynchronize());
    CK(dev_alloc(&t->d_status, sizeof(int)));
    CK(cudaMemsetAsync(t->d_status, 0, sizeof(int), s));

    // 1. FP32 table in the ghost-plane layout
    const size_t f32_bytes = (size_t)t->rows * t->row_stride * sizeof(float);
    float *f32 = nullptr;
    CK(dev_alloc(&f32, f32_bytes));
    const size_t esz = coeffs_is_double ? 8 : 4;
    const size_t src_row_bytes = (size_t)t->Lreal * esz;
    if (coeffs_on_device) {
        cudaError_t e = launch_stage_rows(coeffs, coeffs_is_double, 0, src_rows, t->geo,
                                          t->Lreal, t->row_stride, f32, s);
        if (e != cudaSuccess) { cudaFree(f32); return cuda_fail(e); }
    } else {
        // host source: stream it through a bounded device buffer
        long long slab = std::max<long long>(1, (64LL << 20) / (long long)src_row_bytes);
        slab = std::min(slab, src_rows);
        void *tmp = nullptr;
        cudaError_t e = dev_alloc(&tmp, (size_t)slab * src_row_bytes);
        if (e != cudaSuccess) { cudaFree(f32); return cuda_fail(e); }
        for (long long r0 = 0; r0 < src_rows && e == cudaSuccess; r0 += slab) {
            const long long nr = std::min(slab, src_rows - r0);
            e = cudaMemcpyAsync(tmp, static_cast<const char *>(coeffs) + (size_t)r0 * src_row_bytes,
                                (size_t)nr * src_row_bytes, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = launch_stage_rows(tmp, coeffs_is_double, r0, nr, t->geo, t->Lreal,
                                      t->row_stride, f32, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // tmp is reused
        }
        cudaFree(tmp);
        if (e != cudaSuccess) { cudaFree(f32); return cuda_fail(e); }
    }

    if (t->elem == ELEM_F32) {
        t->d_table = f32;
        t->table_bytes = f32_bytes;
    } else {
        // 2. per-component scales, then quantise
        std::vector<float> ones((size_t)t->row_stride, 1.0f);
        unsigned int *bits = nullptr;
        cudaError_t e = dev_alloc(&t->d_scales, sizeof(float) * (size_t)t->row_stride);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(t->d_scales, ones.data(), sizeof(float) * ones.size(),
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = dev_alloc(&bits, sizeof(unsigned int) * (size_t)t->Lreal);
        if (e == cudaSuccess) e = launch_absmax(f32, t->rows, t->row_stride, t->Lreal, bits, s);
        if (e == cudaSuccess)
            e = launch_make_scales(bits, t->Lreal, t->is_complex ? 1 : 0, t->d_scales, s);
        const size_t qbytes = (size_t)t->rows * t->row_stride * 2;
        if (e == cudaSuccess) e = dev_alloc(&t->d_table, qbytes);
        if (e == cudaSuccess)
            e = launch_quantize(f32, t->rows, t->row_stride, t->Lreal, t->d_scales, t->elem,
                                t->d_table, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (bits) cudaFree(bits);
        cudaFree(f32);
        if (e != cudaSuccess) return cuda_fail(e);
        t->table_bytes = qbytes;
    }
    CK(cudaStreamSynchronize(s));
    return BLIP_OK;
}

}  // namespace

extern "C" {

const char *blip_strerror(int code)
{
    switch (code) {
    case BLIP_OK: return "ok";
    case BLIP_ERR_INVALID_ARG: return "invalid argument";
    case BLIP_ERR_SINGULAR_LATTICE: return "singular lattice";
    case BLIP_ERR_OOM: return "out of memory";
    case BLIP_ERR_CUDA: return "CUDA error";
    case BLIP_ERR_UNSUPPORTED_DTYPE: return "unsupported storage kind";
    case BLIP_ERR_NO_DEVICE: return "no sm_103 CUDA device";
    case BLIP_ERR_SCRATCH_LIMIT:
        return "batch needs more sort scratch than the fixed no-allocation buffer holds";
    default: return "unknown error";
    }
}

int blip_last_cuda_error(void) { return g_last_cuda_error; }

int blip_create(const int grid[3], const double lattice[9], int n_orb, int storage, int norm,
                const void *coeffs, int coeffs_is_double, int coeffs_on_device, blip_table *out)
{
    if (!out) return BLIP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid || !lattice || !coeffs || n_orb < 1) return BLIP_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (grid[a] < 4 || grid[a] > (1 << 20)) return BLIP_ERR_INVALID_ARG;
    if ((long long)grid[0] * grid[1] * (grid[2] + 3) >= (1LL << 31)) return BLIP_ERR_INVALID_ARG;
    for (int i = 0; i < 9; ++i)
        if (!isfinite(lattice[i])) return BLIP_ERR_INVALID_ARG;
    if (storage < BLIP_F32 || storage > BLIP_BF16PAIR) return BLIP_ERR_UNSUPPORTED_DTYPE;
    if (norm != BLIP_NORM_BSPLINE && norm != BLIP_NORM_ALFE_GILLAN) return BLIP_ERR_INVALID_ARG;
    if (n_orb > (1 << 24)) return BLIP_ERR_INVALID_ARG;
    blip_table_s *t = new (std::nothrow) blip_table_s();
    if (!t) return BLIP_ERR_OOM;
    int rc = create_impl(grid, lattice, n_orb, storage, norm, coeffs, coeffs_is_double,
                         coeffs_on_device, t);
    if (rc != BLIP_OK) {
        free_table(t);
        return rc;
    }
    *out = t;
    return BLIP_OK;
}

int blip_destroy(blip_table t)
{
    if (!t) return BLIP_OK;
    if (t->used) {
        cudaStreamSynchronize(t->last_stream);
    }
    free_table(t);
    return BLIP_OK;
}

int blip_eval(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
              int n_walkers, void *values, void *grads, void *laps, void *stream)
{
    int rc = validate_eval(t, pos, n_elec, walker_offsets, n_walkers, values, grads, laps);
    if (rc) return rc;
    return eval_device(t, pos, n_elec, walker_offsets, n_walkers, values, grads, laps,
                       static_cast<cudaStream_t>(stream), pick(t, n_elec, grads == nullptr));
}

int blip_probe_gather(blip_table t, const double *pos, int n_elec, void *values, void *grads,
                      void *laps, int store_outputs, void *stream)
{
    if (!t || n_elec < 0 || (n_elec > 0 && !pos)) return BLIP_ERR_INVALID_ARG;
    if (store_outputs && n_elec > 0 && (!values || !grads || !laps)) return BLIP_ERR_INVALID_ARG;
    if (t->elem != ELEM_F32) return BLIP_ERR_UNSUPPORTED_DTYPE;
    if (n_elec == 0) return BLIP_OK;
    const KernelChoice kc{VAR_REGISTER_PERSIST, 1, 8, 0};
    EvalParams p = make_params(t, pos, n_elec, nullptr, 0, store_outputs ? values : nullptr,
                               store_outputs ? grads : nullptr, store_outputs ? laps : nullptr, kc);
    p.n_k = 0;                       // the phases are arithmetic the probe leaves out
    CK(launch_probe(p, kc.warps, t->sm_count, store_outputs != 0, static_cast<cudaStream_t>(stream)));
    t->last_stream = static_cast<cudaStream_t>(stream);
    t->used = true;
    return BLIP_OK;
}

// Device address of a pinned (page-locked) host buffer, or nullptr if p is
// ordinary pageable memory.
void *mapped_device_ptr(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int blip_eval_host(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
                   int n_walkers, void *values, void *grads, void *laps)
{
    int rc = validate_eval(t, pos, n_elec, walker_offsets, n_walkers, values, grads, laps);
    if (rc) return rc;
    if (n_elec == 0) return BLIP_OK;
    // Pinned host buffers: the kernel reads the positions and writes the
    // outputs across the host link itself (zero-copy), so the transfers
    // overlap the table gather instead of following it.
    {
        void *dp = mapped_device_ptr(pos), *dv = mapped_device_ptr(values);
        void *dg = grads ? mapped_device_ptr(grads) : nullptr;
        void *dl = laps ? mapped_device_ptr(laps) : nullptr;
        void *doff = walker_offsets ? mapped_device_ptr(walker_offsets) : nullptr;
        if (dp && dv && (!grads || (dg && dl)) && (!walker_offsets || doff)) {
            rc = eval_device(t, static_cast<const double *>(dp), n_elec,
                             static_cast<const int *>(doff), n_walkers, dv, dg, dl,
                             t->own_stream, pick(t, n_elec, grads == nullptr));
            if (rc) return rc;
            CK(cudaStreamSynchronize(t->own_stream));
            return BLIP_OK;
        }
    }
    const size_t L = (size_t)t->Lreal;
    const size_t pos_b = (size_t)n_elec * 3 * sizeof(double);
    const size_t off_b = walker_offsets ? (size_t)(n_walkers + 1) * sizeof(int) : 0;
    const size_t val_b = (size_t)n_elec * L * sizeof(float);
    const size_t out_b = grads ? 5 * val_b : val_b;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    rc = grow_stage(t, up(pos_b) + up(off_b) + out_b);
    if (rc) return rc;
    char *base = static_cast<char *>(t->stage);
    double *d_pos = reinterpret_cast<double *>(base);
    int *d_off = walker_offsets ? reinterpret_cast<int *>(base + up(pos_b)) : nullptr;
    float *d_val = reinterpret_cast<float *>(base + up(pos_b) + up(off_b));
    float *d_grd = grads ? d_val + (size_t)n_elec * L : nullptr;
    float *d_lap = grads ? d_grd + (size_t)n_elec * 3 * L : nullptr;
    cudaStream_t s = t->own_stream;
    CK(cudaMemcpyAsync(d_pos, pos, pos_b, cudaMemcpyHostToDevice, s));
    if (d_off) CK(cudaMemcpyAsync(d_off, walker_offsets, off_b, cudaMemcpyHostToDevice, s));
    rc = eval_device(t, d_pos, n_elec, d_off, n_walkers, d_val, d_grd, d_lap, s,
                     pick(t, n_elec, grads == nullptr));
    if (rc) return rc;
    CK(cudaMemcpyAsync(values, d_val, val_b, cudaMemcpyDeviceToHost, s));
    if (grads) {
        CK(cudaMemcpyAsync(grads, d_grd, 3 * val_b, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(laps, d_lap, val_b, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return BLIP_OK;
}

int blip_status(blip_table t, int *device_status)
{
    if (!t || !device_status) return BLIP_ERR_INVALID_ARG;
    if (t->used) CK(cudaStreamSynchronize(t->last_stream));
    int h = 0;
    CK(cudaMemcpy(&h, t->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(t->d_status, 0, sizeof(int)));
    *device_status = h;
    return BLIP_OK;
}

int blip_info(blip_table t, long long out[8])
{
    if (!t || !out) return BLIP_ERR_INVALID_ARG;
    out[0] = t->rows;
    out[1] = t->row_stride;
    out[2] = t->Lreal;
    out[3] = elem_bytes(t->elem);
    out[4] = (long long)t->table_bytes;
    out[5] = t->storage;
    out[6] = t->sm_count;
    out[7] = t->auto_mode ? VAR_AUTO : t->choice.variant;
    return BLIP_OK;
}

int blip_set_kernel(blip_table t, int variant, int chunks, int warps, int sort)
{
    if (!t) return BLIP_ERR_INVALID_ARG;
    if (variant == VAR_AUTO) {
        t->auto_mode = true;
        return BLIP_OK;
    }
    if (variant == VAR_SPLIT) {
        // one chunk per item, 4 warps per block; no Bloch epilogue
        if (t->n_k || chunks != 1 || warps != 4) return BLIP_ERR_INVALID_ARG;
    } else if (variant == VAR_REGISTER_PIPE3) {
        // two batches in flight: FP32 tables, one chunk per warp
        if (t->elem != ELEM_F32 || chunks != 1) return BLIP_ERR_INVALID_ARG;
        if (warps < 1 || warps > 16) return BLIP_ERR_INVALID_ARG;
    } else if (variant == VAR_REGISTER_PERSIST) {
        // as 9, resident warps; no Bloch epilogue
        if (t->elem != ELEM_F32 || chunks != 1 || t->n_k) return BLIP_ERR_INVALID_ARG;
        if (warps < 1 || warps > 16) return BLIP_ERR_INVALID_ARG;
    } else if (variant == VAR_REGISTER || variant == VAR_REGISTER_PIPE || variant == VAR_REGISTER_ROLLED ||
        variant == VAR_REGISTER_L1 || variant == VAR_REGISTER_LOCKSTEP) {
        const int max_chunks = t->elem == ELEM_F32 ? 3 : 1;
        if (chunks < 1 || chunks > max_chunks) return BLIP_ERR_INVALID_ARG;
        if (warps < 1 || warps > 16) return BLIP_ERR_INVALID_ARG;
    } else if (variant == VAR_GROUPED) {
        // chunks = electrons per group (2 or 4); always evaluated in cell order
        if ((chunks != 2 && chunks != 4) || warps < 1 || warps > 8) return BLIP_ERR_INVALID_ARG;
        sort = 1;
    } else if (variant == VAR_STAGED) {
        // chunks = tile cells along a_3 (2 or 4); warps = consumer warps per CTA
        if (t->n_k) return BLIP_ERR_INVALID_ARG;          // no Bloch epilogue in this kernel
        if ((chunks != 2 && chunks != 4) || (warps != 12 && warps != 16)) return BLIP_ERR_INVALID_ARG;
        sort = 1;
    } else if (variant == VAR_TENSOR) {
        // one configuration; always evaluated in cell order; no Bloch epilogue
        if (t->n_k || chunks != 1 || warps != 1) return BLIP_ERR_INVALID_ARG;
        sort = 1;
        const int rc = tc_prepare(t);
        if (rc) return rc;
    } else if (variant == VAR_BULK) {
        if (t->n_k) return BLIP_ERR_INVALID_ARG;          // no Bloch epilogue in this kernel
        // chunks = consumer warps per CTA (chunks per tile), warps = pipeline stages
        if (chunks < 1 || chunks > 8 || warps < 2 || warps > 32) return BLIP_ERR_INVALID_ARG;
        if (bulk_smem_bytes(chunks, warps) > 227 * 1024) return BLIP_ERR_INVALID_ARG;
    } else {
        return BLIP_ERR_INVALID_ARG;
    }
    // sort 2: sorted, and the register kernels' items ordered chunk group
    // slowest
    const bool order_ok = variant == VAR_REGISTER || variant == VAR_REGISTER_PIPE ||
                          variant == VAR_REGISTER_ROLLED || variant == VAR_REGISTER_PIPE3 ||
                          variant == VAR_REGISTER_PERSIST;
    if (sort != 0 && sort != 1 && !(sort == 2 && order_ok)) return BLIP_ERR_INVALID_ARG;
    t->auto_mode = false;
    t->choice = KernelChoice{variant, chunks, warps, sort};
    return BLIP_OK;
}

int blip_autotune(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
                  int n_walkers, void *values, void *grads, void *laps, void *stream,
                  int chosen[4])
{
    int rc = validate_eval(t, pos, n_elec, walker_offsets, n_walkers, values, grads, laps);
    if (rc) return rc;
    if (n_elec == 0) return BLIP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<KernelChoice> cands;
    const int max_chunks = t->elem == ELEM_F32 ? 3 : 1;
    std::vector<int> tws;
    for (int d : {1, 2, 3, 4, 6})
        tws.push_back(std::min(8, (t->nchunk + d - 1) / d));
    std::sort(tws.begin(), tws.end());
    tws.erase(std::unique(tws.begin(), tws.end()), tws.end());
    for (int srt = 0; srt <= (n_elec >= 4096 ? 1 : 0); ++srt) {
        for (int c = 1; c <= max_chunks; ++c)
            for (int w : {4, 8, 16}) {
                cands.push_back(KernelChoice{VAR_REGISTER, c, w, srt});
                cands.push_back(KernelChoice{VAR_REGISTER_PIPE, c, w, srt});
                cands.push_back(KernelChoice{VAR_REGISTER_ROLLED, c, w, srt});
                if (c == 1 && t->elem == ELEM_F32) {
                    // the persistent form first: near-ties go to it
                    if (!t->n_k) {
                        cands.push_back(KernelChoice{VAR_REGISTER_PERSIST, c, w, srt});
                        if (srt && t->nchunk > c)
                            cands.push_back(KernelChoice{VAR_REGISTER_PERSIST, c, w, 2});
                    }
                    cands.push_back(KernelChoice{VAR_REGISTER_PIPE3, c, w, srt});
                    if (srt && t->nchunk > c) cands.push_back(KernelChoice{VAR_REGISTER_PIPE3, c, w, 2});
                }
                if (srt && t->nchunk > c) {       // several chunk groups: try their order too
                    cands.push_back(KernelChoice{VAR_REGISTER, c, w, 2});
                    cands.push_back(KernelChoice{VAR_REGISTER_PIPE, c, w, 2});
                    cands.push_back(KernelChoice{VAR_REGISTER_ROLLED, c, w, 2});
                }
                if (srt) cands.push_back(KernelChoice{VAR_REGISTER_L1, c, w, srt});
                if (srt) cands.push_back(KernelChoice{VAR_REGISTER_LOCKSTEP, c, w, srt});
            }
        for (int tw : tws)
            for (int st : {4, 8, 16})
                if (!t->n_k && bulk_smem_bytes(tw, st) <= 227 * 1024)
                    cands.push_back(KernelChoice{VAR_BULK, tw, st, srt});
        if (srt)
            for (int g : {2, 4})
                for (int w : {4, 8}) cands.push_back(KernelChoice{VAR_GROUPED, g, w, 1});
        if (!t->n_k) cands.push_back(KernelChoice{VAR_SPLIT, 1, 4, srt});
        if (srt && !t->n_k)
            for (int tz : {2, 4})
                for (int cw : {12, 16}) cands.push_back(KernelChoice{VAR_STAGED, tz, cw, 1});
        // tensor cores once the batch holds half an electron per cell or more
        const long long cells = (long long)t->grid[0] * t->grid[1] * t->grid[2];
        if (srt && !t->n_k && 2LL * n_elec >= cells && tc_prepare(t) == BLIP_OK)
            cands.push_back(KernelChoice{VAR_TENSOR, 1, 1, 1});
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // Each configuration is timed from a cold L2 (a read sweep of a 256 MB
    // scratch, twice the L2, before every run, outside the timed window, so
    // that L2 holds only clean lines), as it runs in a Monte Carlo step
    // between other work.  Three passes: every candidate once (after one
    // untimed run; median of 3 if under 0.2 ms); the 16 fastest of those,
    // median of 7 runs; the ones
    // within 5 % of the best median (at most 4), 15 more runs each,
    // interleaved.  The last pass keeps the earliest candidate of the list
    // whose median is within 1 % of the best, so that configurations whose
    // gap is below the timing noise do not trade places from run to run.
    void *flush = nullptr;
    const size_t flush_bytes = 256u << 20;
    if (dev_alloc(&flush, flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        flush = nullptr;                   // no room: time with a warm L2
    }
    // one timed run of configuration kc from a cold L2, in ms
    auto timed_run = [&](const KernelChoice &kc, float &ms) -> int {
        if (flush) launch_l2_sweep(flush, flush_bytes, t->sm_count, s);
        cudaEventRecord(e0, s);
        int r = eval_device(t, pos, n_elec, walker_offsets, n_walkers, values, grads, laps, s, kc);
        cudaEventRecord(e1, s);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) return cuda_fail(ce);
        cudaEventElapsedTime(&ms, e0, e1);
        return r;
    };
    typedef std::pair<float, size_t> Timed;   // (ms, index into cands)
    auto by_time = [](const Timed &a, const Timed &b) {
        return a.first < b.first || (a.first == b.first && a.second < b.second);
    };
    // first pass: every candidate once (median of 3 for launches under
    // 0.2 ms, whose single timings scatter by more than their gaps)
    std::vector<Timed> once;
    for (size_t i = 0; i < cands.size() && rc == 0; ++i) {
        rc = eval_device(t, pos, n_elec, walker_offsets, n_walkers, values, grads, laps, s,
                         cands[i]);
        float ms[3] = {0.0f, 0.0f, 0.0f};
        if (rc == 0) rc = timed_run(cands[i], ms[0]);
        if (rc == 0 && ms[0] < 0.2f) {
            for (int rep = 1; rep < 3 && rc == 0; ++rep) rc = timed_run(cands[i], ms[rep]);
            std::sort(ms, ms + 3);
            ms[0] = ms[1];
        }
        if (rc == 0) once.push_back({ms[0], i});
    }
    // second pass: the 16 fastest, median of 7
    std::vector<Timed> med;
    if (rc == 0) {
        std::sort(once.begin(), once.end(), by_time);
        for (size_t j = 0; j < once.size() && j < 16 && rc == 0; ++j) {
            float ts[7];
            for (int rep = 0; rep < 7 && rc == 0; ++rep) rc = timed_run(cands[once[j].second], ts[rep]);
            if (rc) break;
            std::sort(ts, ts + 7);
            med.push_back({ts[3], once[j].second});
        }
    }
    KernelChoice bestc = cands[0];
    if (rc == 0) {
        // third pass: the candidates within 5 % of the best median, 15 more
        // runs each, interleaved so that slow drifts of the clock hit all of
        // them alike
        std::sort(med.begin(), med.end(), by_time);
        std::vector<size_t> fin;
        for (const auto &m : med)
            if (m.first <= 1.05f * med[0].first && fin.size() < 4) fin.push_back(m.second);
        std::sort(fin.begin(), fin.end());        // list order, for the tie-break
        std::vector<std::vector<float>> ts(fin.size());
        for (int rep = 0; rep < 15 && rc == 0 && fin.size() > 1; ++rep)
            for (size_t i = 0; i < fin.size() && rc == 0; ++i) {
                float ms = 0.0f;
                rc = timed_run(cands[fin[i]], ms);
                ts[i].push_back(ms);
            }
        bestc = cands[med[0].second];
        if (rc == 0 && fin.size() > 1) {
            std::vector<float> m(fin.size());
            float best = 1e30f;
            for (size_t i = 0; i < fin.size(); ++i) {
                std::sort(ts[i].begin(), ts[i].end());
                m[i] = ts[i][ts[i].size() / 2];
                best = std::min(best, m[i]);
            }
            for (size_t i = 0; i < fin.size(); ++i)
                if (m[i] <= 1.01f * best) {
                    bestc = cands[fin[i]];
                    break;
                }
        }
    }
    if (flush) cudaFree(flush);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    t->tuned[tune_key(n_elec, grads == nullptr)] = bestc;
    t->auto_mode = true;
    if (chosen) {
        chosen[0] = bestc.variant;
        chosen[1] = bestc.chunks;
        chosen[2] = bestc.warps;
        chosen[3] = bestc.sort;
    }
    return BLIP_OK;
}

int blip_set_l2_residency(blip_table t, double fraction)
{
    if (!t || !(fraction >= 0.0) || fraction > 1.0) return BLIP_ERR_INVALID_ARG;
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != t->device) return BLIP_ERR_INVALID_ARG;
    if (fraction == 0.0) {
        if (t->l2_limit_set) {
            if (t->used) CK(cudaStreamSynchronize(t->last_stream));
            CK(cudaCtxResetPersistingL2Cache());
            CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0));
            t->l2_limit_set = false;
        }
        t->l2_window = 0;
        return BLIP_OK;
    }
    int max_persist = 0, max_window = 0;
    CK(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev));
    CK(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev));
    if (max_persist <= 0 || max_window <= 0) return BLIP_ERR_INVALID_ARG;
    const size_t want = (size_t)(fraction * (double)t->table_bytes);
    const size_t window = std::min(want, (size_t)max_window);
    const size_t limit = std::min(window, (size_t)max_persist);
    CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, limit));
    t->l2_limit_set = true;
    t->l2_window = window;
    // more window than persisting lines: mark only a share of it persisting
    t->l2_hit_ratio = window > 0 ? std::min(1.0f, (float)((double)limit / (double)window)) : 1.0f;
    return BLIP_OK;
}

int blip_probe_l2_read(const void *buf, size_t bytes, int reps, void *stream)
{
    if (!buf || bytes < 16 || bytes % 16 || ((uintptr_t)buf & 15u) || reps < 1)
        return BLIP_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(launch_l2_read(buf, bytes, reps, sms, static_cast<cudaStream_t>(stream)));
    return BLIP_OK;
}

int blip_test_fail_alloc(int n)
{
    g_alloc_fail_after.store(n < 0 ? -1 : n);
    return BLIP_OK;
}

int blip_test_stall_pipeline(blip_table t, int on)
{
    if (!t) return BLIP_ERR_INVALID_ARG;
    t->test_stall = on ? 1 : 0;
    return BLIP_OK;
}

int blip_sm_update(int n_walkers, int n, float *dinv, const float *rows, const int *cols,
                   float *work, void *stream)
{
    if (n_walkers < 0 || n < 1 || n > (1 << 15)) return BLIP_ERR_INVALID_ARG;
    if (n_walkers == 0) return BLIP_OK;
    if (!dinv || !rows || !cols || !work) return BLIP_ERR_INVALID_ARG;
    if (n_walkers > 65535) return BLIP_ERR_INVALID_ARG;     // grid y/z limit
    CK(launch_sm_update(n_walkers, n, dinv, rows, cols, work, static_cast<cudaStream_t>(stream)));
    return BLIP_OK;
}

int blip_set_kpoints(blip_table t, int n_k, const double *kfrac, const int *koffs)
{
    if (!t) return BLIP_ERR_INVALID_ARG;
    if (n_k == 0) {
        t->n_k = 0;
        return BLIP_OK;
    }
    if (!t->is_complex) return BLIP_ERR_UNSUPPORTED_DTYPE;
    if (n_k < 0 || n_k > kMaxKpoints || !kfrac || !koffs) return BLIP_ERR_INVALID_ARG;
    if (koffs[0] != 0 || koffs[n_k] != t->n_orb) return BLIP_ERR_INVALID_ARG;
    for (int q = 0; q < n_k; ++q) {
        if (koffs[q + 1] < koffs[q]) return BLIP_ERR_INVALID_ARG;
        for (int c = 0; c < 3; ++c)
            if (!isfinite(kfrac[3 * q + c])) return BLIP_ERR_INVALID_ARG;
    }
    // k_q = 2 pi A^{-T} kappa_q: component c = 2 pi sum_a kappa_a (A^{-1})_{a c}
    const double two_pi = 6.283185307179586;
    for (int q = 0; q < n_k; ++q)
        for (int c = 0; c < 3; ++c) {
            double k = 0.0;
            for (int a = 0; a < 3; ++a) k += kfrac[3 * q + a] * t->geo.ainv[3 * a + c];
            t->kcart[q][c] = (float)(two_pi * k);
            t->kfrac[q][c] = kfrac[3 * q + c];
        }
    for (int q = 0; q <= n_k; ++q) t->koff[q] = koffs[q];
    t->n_k = n_k;
    if (!has_bloch_epilogue(t->choice)) t->choice = KernelChoice{VAR_REGISTER, 1, 8, 0};
    for (auto &kv : t->tuned)
        if (!has_bloch_epilogue(kv.second)) kv.second = KernelChoice{VAR_REGISTER, 1, 8, 0};
    return BLIP_OK;
}

int blip_eval_ratio(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
                    int n_walkers, const float *inv_cols, float *ratio, float *values, int sort,
                    void *stream)
{
    if (!t || n_elec < 0 || (walker_offsets && n_walkers < 1)) return BLIP_ERR_INVALID_ARG;
    if (n_elec > 0 && (!pos || !inv_cols || !ratio)) return BLIP_ERR_INVALID_ARG;
    if (t->is_complex) return BLIP_ERR_UNSUPPORTED_DTYPE;
    if (sort < 0 || sort > 2) return BLIP_ERR_INVALID_ARG;
    if (n_elec == 0) return BLIP_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EvalParams p{};
    p.table = t->d_table;
    p.scales = t->d_scales;
    p.row_stride = t->row_stride;
    p.Lreal = t->Lreal;
    p.nchunk = t->nchunk;
    p.groups = 1;
    p.items = n_elec;
    p.geo = t->geo;
    p.pos = pos;
    p.n_elec = n_elec;
    p.perm = nullptr;
    if (sort) {
        int *perm = nullptr;
        const ElecGeo *rec = nullptr;
        int rc = sorted_order(t, pos, n_elec, s, &perm, &rec);
        if (rc) return rc;
        p.perm = perm;
        p.georec = rec;
    }
    p.offsets = walker_offsets;
    p.n_walkers = walker_offsets ? n_walkers : 0;
    p.values = values;
    p.grads = nullptr;
    p.laps = nullptr;
    p.vec_out = 0;
    p.status = t->d_status;
    // dense batches (at least one electron per two cells) in cell order go
    // to the tensor cores; the operand planes and tensor maps are made on
    // first use, outside stream capture
    bool tc = false;
    if (sort == 1 && 2LL * n_elec >= (long long)t->grid[0] * t->grid[1] * t->grid[2]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(s, &cs));
        if (t->tc_ready || cs == cudaStreamCaptureStatusNone) {
            const int rc = tc_prepare(t);
            if (rc != BLIP_OK && rc != BLIP_ERR_INVALID_ARG) return rc;
            tc = rc == BLIP_OK;
        }
    }
    // the ratio kernel's per-electron column scales (FP16 operands)
    if (tc && !values && t->elem != ELEM_BF16 && t->rsig_n < n_elec) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusNone) {
            if (t->d_rsig) cudaFree(t->d_rsig);
            t->d_rsig = nullptr;
            t->rsig_n = 0;
            CK(dev_alloc(&t->d_rsig, sizeof(float) * (size_t)n_elec));
            t->rsig_n = n_elec;
        }
    }
    if (tc && !values && (t->elem == ELEM_BF16 || t->rsig_n >= n_elec)) {
        // the orbital sum on the tensor cores, inverse columns as an operand
        const int *keys = nullptr, *cell_end = nullptr;
        sort_views(t->geo, n_elec, t->scratch, &keys, &cell_end);
        if (t->elem == ELEM_F32) p.scales = t->d_tc_scales;   // the planes' power-of-two scales
        CK(launch_ratio_tc(p, t->elem, cell_end, t->d_cols, t->ncols, t->rows, t->tc_tmap,
                           t->tc_wide ? &t->tc_tmap5k : nullptr, t->d_tc_ctr, t->sm_count,
                           t->test_stall, s, inv_cols, ratio, t->d_rsig));
    } else if (tc) {
        const int *keys = nullptr, *cell_end = nullptr;
        sort_views(t->geo, n_elec, t->scratch, &keys, &cell_end);
        if (t->elem == ELEM_F32) p.scales = t->d_tc_scales;   // the planes' power-of-two scales
        CK(launch_tc(p, t->elem, cell_end, t->d_cols, t->ncols, t->rows, t->tc_tmap,
                     t->tc_wide ? &t->tc_tmap5 : nullptr, t->d_tc_ctr, t->sm_count,
                     t->test_stall, s, inv_cols, ratio));
    } else {
        CK(launch_ratio(p, t->elem, inv_cols, ratio, 4, s));
    }
    t->last_stream = s;
    t->used = true;
    return BLIP_OK;
}

int blip_graph_create(blip_table t, const double *pos, int n_elec, const int *walker_offsets,
                      int n_walkers, void *values, void *grads, void *laps, int per_launch,
                      blip_graph *out)
{
    if (!out) return BLIP_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = validate_eval(t, pos, n_elec, walker_offsets, n_walkers, values, grads, laps);
    if (rc) return rc;
    if (n_elec < 1 || per_launch < 1) return BLIP_ERR_INVALID_ARG;
    blip_graph_s *g = new (std::nothrow) blip_graph_s();
    if (!g) return BLIP_ERR_OOM;
    g->table = t;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete g; return cuda_fail(e); }
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    const size_t L = (size_t)t->Lreal;
    for (int e0 = 0; e0 < n_elec && e == cudaSuccess && rc == 0; e0 += per_launch) {
        const int ne = std::min(per_launch, n_elec - e0);
        const bool whole = (e0 == 0 && ne == n_elec);
        rc = eval_device(t, pos + 3 * (size_t)e0, ne, whole ? walker_offsets : nullptr, n_walkers,
                         static_cast<float *>(values) + (size_t)e0 * L,
                         grads ? static_cast<float *>(grads) + (size_t)e0 * 3 * L : nullptr,
                         laps ? static_cast<float *>(laps) + (size_t)e0 * L : nullptr, s,
                         pick(t, ne, grads == nullptr));
    }
    cudaError_t ee = cudaStreamEndCapture(s, &g->graph);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess && rc == 0) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    cudaStreamDestroy(s);
    t->last_stream = nullptr;
    if (e != cudaSuccess || rc != 0) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc ? rc : cuda_fail(e);
    }
    *out = g;
    return BLIP_OK;
}

int blip_graph_launch(blip_graph g, void *stream)
{
    if (!g || !g->exec) return BLIP_ERR_INVALID_ARG;
    CK(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
    g->table->last_stream = static_cast<cudaStream_t>(stream);
    g->table->used = true;
    return BLIP_OK;
}

int blip_graph_destroy(blip_graph g)
{
    if (!g) return BLIP_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return BLIP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Evaluation without any allocation: the sorted evaluation path with its sort
// scratch taken from a fixed device array compiled into this library.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;   // 8 MiB per device
constexpr int kNoAllocMaxDevices = 64;

// The fixed scratch buffer.  Every device that loads this library holds one
// copy until the process exits.  Host code must not use this name as an
// address: it is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the fixed buffer on the current device, looked up once
// per device (the first call may load this library's module on that device).
int noalloc_scratch(void **out)
{
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return BLIP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return BLIP_OK;
}

}  // namespace

extern "C" int blip_eval_sorted_noalloc(blip_table t, const double *pos, int n_elec,
                                        const int *walker_offsets, int n_walkers, void *values,
                                        void *grads, void *laps, void *stream)
{
    int rc = validate_eval(t, pos, n_elec, walker_offsets, n_walkers, values, grads, laps);
    if (rc) return rc;
    if (n_elec == 0) return BLIP_OK;
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != t->device) return BLIP_ERR_INVALID_ARG;      // the table's device must be current
    if (sort_scratch_bytes(n_elec, t->geo) > kNoAllocScratchBytes) return BLIP_ERR_SCRATCH_LIMIT;
    void *scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const KernelChoice kc = pick(t, n_elec, grads == nullptr);
    if (t->n_k && !has_bloch_epilogue(kc)) return BLIP_ERR_INVALID_ARG;
    // the sort clears its histogram itself and overwrites everything else it
    // reads; no per-electron records (the kernels wrap the positions)
    int *perm = nullptr;
    CK(launch_sort(t->geo, pos, n_elec, scratch, &perm, s));
    EvalParams p = make_params(t, pos, n_elec, walker_offsets, n_walkers, values, grads, laps, kc);
    p.perm = perm;
    return launch_choice(t, p, kc, scratch, s);
}

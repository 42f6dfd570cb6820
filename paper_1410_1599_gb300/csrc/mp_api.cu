// mp_api.cu -- the C ABI of libmpgemm.so (include/mpgemm.h): argument checks,
// dispatch to the word-capacity class, the breadth-first Strassen/Winograd
// driver (arXiv 1410.1599 Sec. 2) and the device status word.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/mpgemm.h"
#include "mp_internal.h"

using namespace mpg;

namespace {

struct ThreadState {
    cudaStream_t stream = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int odd_policy = MP_PEEL;
    int lu_panel = 128, lu_algo = MP_SIMPLE, lu_cutoff = 64;
    bool lu_pivoting = true;
    bool split_truncate = true;
    bool leaf_tma = true;
    long long singular_col = -1;
    long long split_fallbacks = 0;
};
thread_local ThreadState g_ts;

// A second stream per thread and device for work that can overlap the main
// stream's (the peeled border products of the recursion), with the events
// that fork it from and join it back to the main stream.  Created on first
// use and kept for the thread's lifetime.
struct SideStream {
    int device = -1;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
thread_local std::vector<SideStream> g_side;

SideStream *side_stream()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    for (SideStream &x : g_side)
        if (x.device == dev) return &x;
    SideStream x;
    x.device = dev;
    if (cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    g_side.push_back(x);
    return &g_side.back();
}

std::mutex g_status_mu;
std::vector<DevStatus *> g_status;   // one per device

DevStatus *status_ptr()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if ((int)g_status.size() <= dev) g_status.resize(dev + 1, nullptr);
    if (!g_status[dev]) {
        DevStatus *p = nullptr;
        if (cudaMalloc(&p, sizeof(DevStatus)) != cudaSuccess) return nullptr;
        DevStatus init{0u, 0u, INT64_MAX, 0ull};
        cudaMemcpy(p, &init, sizeof init, cudaMemcpyHostToDevice);
        g_status[dev] = p;
    }
    return g_status[dev];
}

int limbs_of(int p) { return (p + 63) / 64; }

// word-capacity class: smallest W in {4, 8, 16, 32, 64, BIG_W} with 32 W >= 64 L
int wclass(int p)
{
    const int L = limbs_of(p);
    if (L <= 2) return 4;
    if (L <= 4) return 8;
    if (L <= 8) return 16;
    if (L <= 16) return 32;
    if (L <= 32) return 64;
    return mpg::BIG_W;
}

template <typename F>
void dispatch(int p, F &&f)
{
    switch (wclass(p)) {
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 16: f(std::integral_constant<int, 16>{}); break;
    case 32: f(std::integral_constant<int, 32>{}); break;
    case 64: f(std::integral_constant<int, 64>{}); break;
    default: f(std::integral_constant<int, mpg::BIG_W>{}); break;
    }
}

// the classes up to 2048 bits only (exact and split kernels); callers reject
// wider precisions first
template <typename F>
void dispatch_narrow(int p, F &&f)
{
    switch (wclass(p)) {
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 16: f(std::integral_constant<int, 16>{}); break;
    case 32: f(std::integral_constant<int, 32>{}); break;
    default: f(std::integral_constant<int, 64>{}); break;
    }
}

bool valid_prec(int p) { return p >= MP_PREC_MIN && p <= MP_PREC_MAX; }

// checks a caller matrix of the given shape; empty matrices need no pointers
bool valid_mat(const mpmat_t *M, int64_t rows, int64_t cols, int prec)
{
    if (!M || M->prec != prec || M->reserved != 0) return false;
    if (M->rows != rows || M->cols != cols || rows < 0 || cols < 0) return false;
    if (rows == 0 || cols == 0) return true;
    if (M->ld < cols || M->plane < (rows - 1) * M->ld + cols) return false;
    if (!M->limb || !M->exp || !M->sign) return false;
    return true;
}

BMat bmat(const mpmat_t *M)
{
    return BMat{M->limb, M->exp, M->sign, M->ld, M->plane, 0, 0};
}

// [lo, hi) byte ranges of a matrix's three arrays
struct Range { uintptr_t lo, hi; };
void ranges(const mpmat_t *M, Range out[3])
{
    const int L = limbs_of(M->prec);
    const int64_t span = (M->rows - 1) * M->ld + M->cols;
    out[0] = {(uintptr_t)M->limb, (uintptr_t)(M->limb + (int64_t)(L - 1) * M->plane + span)};
    out[1] = {(uintptr_t)M->exp, (uintptr_t)(M->exp + span)};
    out[2] = {(uintptr_t)M->sign, (uintptr_t)(M->sign + span)};
}

bool overlaps(const mpmat_t *X, const mpmat_t *Y)
{
    if (X->rows == 0 || X->cols == 0 || Y->rows == 0 || Y->cols == 0) return false;
    Range a[3], b[3];
    ranges(X, a);
    ranges(Y, b);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (a[i].lo < b[j].hi && b[j].lo < a[i].hi) return true;
    return false;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? MP_OK : MP_ERR_CUDA; }

// ------------------------------------------------------------------ tracing
struct ProfRec { int cls; cudaEvent_t a, b; double units; };
struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    int64_t launches[MP_K_COUNT] = {};
    double ms[MP_K_COUNT] = {}, units[MP_K_COUNT] = {};

    cudaEvent_t ev()
    {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    void drain()   // fold finished records into the totals
    {
        for (auto &r : recs) {
            float t = 0.f;
            cudaEventSynchronize(r.b);
            cudaEventElapsedTime(&t, r.a, r.b);
            launches[r.cls] += 1;
            ms[r.cls] += t;
            units[r.cls] += r.units;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
    }
};
Profiler g_prof;

// Bracket one launch: Prof p(cls, units, stream); <launch>;  (destructor records the end)
struct Prof {
    bool on;
    ProfRec rec;
    cudaStream_t s;
    Prof(int cls, double units, cudaStream_t st) : on(g_prof.on), s(st)
    {
        if (!on) return;
        std::lock_guard<std::mutex> lk(g_prof.mu);
        if (g_prof.recs.size() > 4096) g_prof.drain();
        rec = ProfRec{cls, g_prof.ev(), g_prof.ev(), units};
        cudaEventRecord(rec.a, s);
    }
    // the launch turned out to belong to another class (the leaf's staging)
    void reclass(int cls)
    {
        if (on) rec.cls = cls;
    }
    ~Prof()
    {
        if (!on) return;
        std::lock_guard<std::mutex> lk(g_prof.mu);
        cudaEventRecord(rec.b, s);
        g_prof.recs.push_back(rec);
    }
};

int launch_status() { return cuda_status(cudaGetLastError()); }

// ------------------------------------------------------------- workspace
struct Workspace {
    char *base = nullptr;
    size_t size = 0, used = 0;
    bool owned = false;
    cudaStream_t s = nullptr;

    int acquire(size_t bytes, cudaStream_t st)
    {
        s = st;
        size = bytes;
        used = 0;
        if (bytes == 0) return MP_OK;
        if (g_ts.ws && g_ts.ws_bytes >= bytes) {
            base = (char *)g_ts.ws;
            return MP_OK;
        }
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return MP_ERR_NOMEM;
        }
        base = (char *)p;
        owned = true;
        return MP_OK;
    }
    void *take(size_t bytes)
    {
        size_t off = (used + 255) & ~(size_t)255;
        used = off + bytes;
        return base + off;
    }
    size_t mark() const { return used; }
    void reset(size_t m) { used = m; }
    ~Workspace()
    {
        if (owned && base) cudaFreeAsync(base, s);
    }
};

size_t padded(size_t b) { return (b + 255) & ~(size_t)255; }

// ------------------------------------------------- recursion plan (Sec. 2)
struct LevelDims {
    int64_t m, l, n;      // real sizes of every node at this level
    int64_t M, K, N;      // even sizes of the recursive part (pad or peel)
};

int64_t even_dim(int64_t x, int policy)
{
    if (x % 2 == 0) return x;
    if (policy == MP_MIXED && x % 4 == 3) return x + 1;
    return x - 1;
}

std::vector<LevelDims> plan(int64_t m, int64_t l, int64_t n, int cutoff, int policy)
{
    std::vector<LevelDims> lv;
    for (;;) {
        LevelDims d{m, l, n, m, l, n};
        const bool rec = m > cutoff && l > cutoff && n > cutoff;
        if (rec) {
            d.M = even_dim(m, policy);
            d.K = even_dim(l, policy);
            d.N = even_dim(n, policy);
        }
        lv.push_back(d);
        if (!rec) break;
        m = d.M / 2;
        l = d.K / 2;
        n = d.N / 2;
    }
    return lv;   // lv.size() - 1 recursion levels; the last entry is the leaf
}

// The recursion's buffers keep an even row stride (a padding column after
// an odd one), so that the bulk tensor copies of the leaves can address
// them (byte strides in 16-byte units).
int64_t rec_ld(int64_t cols) { return cols + (cols & 1); }

size_t mat_bytes(int64_t count, int64_t rows, int64_t cols, int L)
{
    const size_t e = (size_t)count * (size_t)rows * (size_t)cols;
    return padded(e * 8 * (size_t)L) + padded(e * 8) + padded(e);
}

size_t recursion_bytes(const std::vector<LevelDims> &lv, int L)
{
    size_t total = 0;
    int64_t nodes = 1;
    for (size_t k = 1; k < lv.size(); ++k) {
        nodes *= 7;
        total += mat_bytes(nodes, lv[k].m, rec_ld(lv[k].l), L);
        total += mat_bytes(nodes, lv[k].l, rec_ld(lv[k].n), L);
        total += mat_bytes(nodes, lv[k].m, rec_ld(lv[k].n), L);
    }
    return total + 256;
}

// count matrices of rows x cols, row stride ld (>= cols)
BMat carve(Workspace &ws, int64_t count, int64_t rows, int64_t cols, int L, int64_t ld = 0)
{
    if (ld < cols) ld = cols;
    const size_t e = (size_t)count * (size_t)rows * (size_t)ld;
    BMat b;
    b.limb = (uint64_t *)ws.take(e * 8 * (size_t)L);
    b.exp = (int64_t *)ws.take(e * 8);
    b.sign = (int8_t *)ws.take(e);
    b.ld = ld;
    b.plane = rows * ld;
    b.bs_limb = (int64_t)L * rows * ld;
    b.bs_es = rows * ld;
    return b;
}

__global__ void fill_zero_kernel(BMat C, int64_t rows, int64_t cols, int L)
{
    const int64_t total = rows * cols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / cols, c = t % cols;
        for (int k = 0; k < L; ++k) C.limb[(int64_t)k * C.plane + r * C.ld + c] = 0ull;
        C.exp[r * C.ld + c] = INT64_MIN;
        C.sign[r * C.ld + c] = 0;
    }
}

// The recursion's buffers and plan for one product (Sec. 2), split into
// the phases a grouped run interleaves: operand sums top-down, the leaf
// products, combinations bottom-up.
struct RecState {
    std::vector<LevelDims> lv;
    std::vector<BMat> A, B, C;
    int algo = 0;
    int64_t leaves = 1;
};

// carve the level buffers and run the operand sums of every level (one
// batched launch per side and level)
template <int W>
void rec_down(RecState &r, int algo, const std::vector<LevelDims> &lv, int p, BMat A0, BMat B0, BMat C0,
              Workspace &ws, cudaStream_t s, bool leaf_views = false)
{
    const int L = limbs_of(p);
    const int D = (int)lv.size() - 1;
    r.lv = lv;
    r.algo = algo;
    r.A.assign(D + 1, BMat{});
    r.B.assign(D + 1, BMat{});
    r.C.assign(D + 1, BMat{});
    r.A[0] = A0;
    r.B[0] = B0;
    r.C[0] = C0;
    int64_t nodes = 1;
    for (int k = 1; k <= D; ++k) {
        nodes *= 7;
        r.A[k] = carve(ws, nodes, lv[k].m, lv[k].l, L, rec_ld(lv[k].l));
        r.B[k] = carve(ws, nodes, lv[k].l, lv[k].n, L, rec_ld(lv[k].n));
        r.C[k] = carve(ws, nodes, lv[k].m, lv[k].n, L, rec_ld(lv[k].n));
    }
    r.leaves = nodes;
    nodes = 1;
    for (int k = 0; k < D; ++k) {
        const LevelDims &d = lv[k];
        const bool skip = leaf_views && k == D - 1;   // plain children stay in the parents
        // work units: numbers read (4 quadrants) and written (7 children, or
        // the ones that are not plain quadrants)
        const double rw = 4.0 + (skip ? (algo == MP_WINOGRAD ? 4.0 : 5.0) : 7.0);
        {
            Prof pr(MP_K_OPERANDS, rw * nodes * (d.M / 2) * (d.K / 2), s);
            launch_operands_a<W>(algo, r.A[k], r.A[k + 1], nodes, d.m, d.l, d.M / 2, d.K / 2, p, s, skip);
        }
        {
            Prof pr(MP_K_OPERANDS, rw * nodes * (d.K / 2) * (d.N / 2), s);
            launch_operands_b<W>(algo, r.B[k], r.B[k + 1], nodes, d.l, d.n, d.K / 2, d.N / 2, p, s, skip);
        }
        nodes *= 7;
    }
}

// peeled borders (last row / column of a node with odd m / n, Simple over
// its whole l); they need only the node's operands
template <int W>
bool rec_has_borders(const RecState &r)
{
    for (size_t k = 0; k + 1 < r.lv.size(); ++k)
        if (r.lv[k].M < r.lv[k].m || r.lv[k].N < r.lv[k].n) return true;
    return false;
}
template <int W>
void rec_borders(const RecState &r, int p, DevStatus *st, cudaStream_t s)
{
    const int D = (int)r.lv.size() - 1;
    int64_t nk = 1;
    for (int k = 0; k < D; ++k, nk *= 7) {
        const LevelDims &d = r.lv[k];
        if (!(d.M < d.m || d.N < d.n)) continue;
        const int64_t mr = std::min(d.M, d.m);
        const int64_t cnt = (d.M < d.m ? d.n : 0) + (d.N < d.n ? mr : 0);
        Prof pr(MP_K_FIXUP, (double)nk * cnt * d.l, s);
        launch_border<W>(r.A[k], r.B[k], r.C[k], nk, d.m, d.l, d.n, mr, d.M < d.m, d.N < d.n, p, st, s);
    }
}

// combinations bottom-up, then the rank-1 fix-up of an odd l
template <int W>
void rec_up(const RecState &r, int p, DevStatus *st, cudaStream_t s)
{
    const int D = (int)r.lv.size() - 1;
    int64_t nodes = r.leaves;
    for (int k = D - 1; k >= 0; --k) {
        nodes /= 7;
        const LevelDims &d = r.lv[k];
        const int64_t mr = std::min(d.M, d.m), nr = std::min(d.N, d.n);
        {
            // work units: numbers read (7 child products) and written (4 quadrants)
            Prof pr(MP_K_COMBINE, 11.0 * nodes * (d.M / 2) * (d.N / 2), s);
            launch_combine<W>(r.algo, r.C[k + 1], r.C[k], nodes, d.M / 2, d.N / 2, mr, nr, p, st, s);
        }
        if (d.K < d.l) {
            Prof pr(MP_K_FIXUP, (double)nodes * mr * nr, s);
            launch_rank1<W>(r.A[k], r.B[k], r.C[k], nodes, mr, nr, d.l, p, st, s);
        }
    }
}

// Children of the last level that are plain quadrants of their parent are
// read by the leaves from the parent (LeafViews) instead of being copied:
// Winograd's M2, M3, M7 take A11, A12, A22 and M2, M3, M6 take B11, B21,
// B22; Strassen's P3, P4 take A11, A22 and P2, P5 take B11, B22.  Only
// where the parent's even part lies inside its real rows and columns (the
// peel policy; a zero-padded quadrant has to be materialised).
template <int W>
bool leaf_views_apply(int algo, const std::vector<LevelDims> &lv, LeafViews &v)
{
    if constexpr (W > 64) {                           // the wide class materialises every child
        return false;
    } else {
        const int D = (int)lv.size() - 1;
        if (D < 1) return false;
        const LevelDims &d = lv[D - 1];
        if (d.M > d.m || d.K > d.l || d.N > d.n) return false;
        for (int t = 0; t < 7; ++t) v.qa[t] = v.qb[t] = 0;
        if (algo == MP_WINOGRAD) {
            v.qa[1] = 1; v.qa[2] = 2; v.qa[6] = 4;     // A11, A12, A22
            v.qb[1] = 1; v.qb[2] = 3; v.qb[5] = 4;     // B11, B21, B22
        } else {
            v.qa[2] = 1; v.qa[3] = 4;                  // A11, A22
            v.qb[1] = 1; v.qb[4] = 4;                  // B11, B22
        }
        return true;
    }
}

template <int W>
int run_recursion(int algo, const std::vector<LevelDims> &lv, int p, BMat A0, BMat B0, BMat C0,
                  Workspace &ws, DevStatus *st, cudaStream_t s)
{
    RecState r;
    LeafViews views{};
    bool use_views = leaf_views_apply<W>(algo, lv, views);
    if (use_views && W <= TMA_MAX_W && g_ts.leaf_tma) {
        // With TMA staging, in-place quadrants pay only where the copies can
        // start at them: an odd column offset (the leaf's l on the A side,
        // n on the B side) or an odd row stride of the caller's matrices at
        // the top level would leave the leaves thread-staged; materialised
        // children (even strides) keep the copies, which gains more.
        const int D = (int)lv.size() - 1;
        bool odd = false;
        for (int t = 0; t < 7; ++t) {
            if ((views.qa[t] == 2 || views.qa[t] == 4) && (lv[D].l & 1)) odd = true;
            if ((views.qb[t] == 2 || views.qb[t] == 4) && (lv[D].n & 1)) odd = true;
        }
        if (D == 1 && ((A0.ld | A0.plane | B0.ld | B0.plane) & 1)) odd = true;
        if (odd) use_views = false;
    }
    rec_down<W>(r, algo, lv, p, A0, B0, C0, ws, s, use_views);
    const int D = (int)lv.size() - 1;
    // the borders run on a second stream, overlapping the leaves, and join
    // before the combinations
    const bool any_border = rec_has_borders<W>(r);
    SideStream *ss = any_border ? side_stream() : nullptr;
    const cudaStream_t bs = ss ? ss->s : s;
    if (ss) {
        cudaEventRecord(ss->fork, s);
        cudaStreamWaitEvent(bs, ss->fork, 0);
    }
    if (any_border) rec_borders<W>(r, p, st, bs);
    if (ss) cudaEventRecord(ss->join, bs);
    // leaves: one grouped Block GEMM over all 7^D products
    {
        Prof pr(MP_K_LEAF, (double)r.leaves * lv[D].m * lv[D].l * lv[D].n, s);
        bool tma;
        if (use_views) {
            views.Ap = r.A[D - 1];
            views.Bp = r.B[D - 1];
            views.nodes = r.leaves / 7;
            views.a_rows = lv[D - 1].m;
            views.a_cols = lv[D - 1].l;
            views.b_rows = lv[D - 1].l;
            views.b_cols = lv[D - 1].n;
            tma = launch_gemm_leaf_views<W>(r.A[D], r.B[D], r.C[D], views, r.leaves, lv[D].m, lv[D].l, lv[D].n,
                                            p, st, s, g_ts.leaf_tma);
        } else {
            tma = launch_gemm_block<W>(r.A[D], r.B[D], r.C[D], r.leaves, lv[D].m, lv[D].l, lv[D].n, p, st, s,
                                       g_ts.leaf_tma);
        }
        if (tma) pr.reclass(MP_K_LEAF_TMA);
    }
    if (ss) cudaStreamWaitEvent(s, ss->join, 0);
    rec_up<W>(r, p, st, s);
    return launch_status();
}

// first diagonal of the split form under the current settings
int split_s0(int p, int64_t l, int64_t *ebits)
{
    if (!g_ts.split_truncate) {
        *ebits = -1;
        return 0;
    }
    return split_first_diagonal(p, l, ebits);
}

// split form: digit planes, exponent / spread vectors, diagonal sums (planes
// s0 .. 2S-2), the list of outputs left to the exact kernel and its count
size_t split_ws_bytes(int64_t m, int64_t l, int64_t n, int p)
{
    const size_t S = (size_t)split_digit_count(p), lp = (size_t)split_row_pad(l);
    int64_t eb;
    const size_t s0 = (size_t)split_s0(p, l, &eb);
    return padded(S * m * lp * 2) + padded(S * n * lp * 2) + padded((size_t)m * 8) +
           padded((size_t)n * 8) + padded((size_t)m) + padded((size_t)n) +
           padded((2 * S - 1 - s0) * m * n * 8) + padded((size_t)m * n * 8) + padded(8) + 8 * 256;
}

int run_split(int64_t m, int64_t l, int64_t n, int p, BMat A, BMat B, BMat C, Workspace &ws,
              DevStatus *st, cudaStream_t s)
{
    // The digit planes are read by TMA loads multicast across the CTAs of a
    // cluster; they must be this GPU's own device memory (a caller's
    // workspace on another device, or host / managed memory, is refused
    // before anything is launched).
    if (!on_current_device(ws.base)) return MP_ERR_ARG;
    const size_t mk = ws.mark();
    const size_t S = (size_t)split_digit_count(p), lp = (size_t)split_row_pad(l);
    __half *pa = (__half *)ws.take(S * m * lp * 2);
    __half *pb = (__half *)ws.take(S * n * lp * 2);
    int64_t *ea = (int64_t *)ws.take((size_t)m * 8);
    int64_t *eb = (int64_t *)ws.take((size_t)n * 8);
    uint8_t *wa = (uint8_t *)ws.take((size_t)m);
    uint8_t *wb = (uint8_t *)ws.take((size_t)n);
    int64_t ebits;
    const int s0 = split_s0(p, l, &ebits);
    long long *D = (long long *)ws.take((2 * S - 1 - (size_t)s0) * m * n * 8);
    int64_t *list = (int64_t *)ws.take((size_t)m * n * 8);
    unsigned long long *count = (unsigned long long *)ws.take(8);
    if (cudaMemsetAsync(count, 0, 8, s) != cudaSuccess) {
        ws.reset(mk);
        return MP_ERR_CUDA;
    }
    {
        Prof pr(MP_K_SPLIT_AUX, (double)(m * l + l * n), s);
        dispatch_narrow(p, [&](auto w) {
            launch_split_prep<decltype(w)::value>(A, B, m, l, n, p, pa, pb, ea, eb, wa, wb, s);
        });
    }
    {
        double pairs = 0;                                   // digit pairs on the kept diagonals
        for (int d = s0; d <= 2 * (int)S - 2; ++d) pairs += std::min<int>(d + 1, 2 * (int)S - 1 - d);
        Prof pr(MP_K_SPLIT, pairs * m * (double)lp * n, s);
        const int rs = launch_split_slices(pa, pb, m, l, n, p, s0, D, st, s);
        if (rs != MP_OK) {
            ws.reset(mk);
            return rs;
        }
    }
    {
        Prof pr(MP_K_SPLIT_AUX, (double)m * n, s);
        dispatch_narrow(p, [&](auto w) {
            launch_split_finish<decltype(w)::value>(D, m, n, p, s0, ebits, ea, eb, wa, wb, C, list, count, st, s);
        });
    }
    if (ebits >= 0) {
        Prof pr(MP_K_SPLIT_AUX, 0.0, s);
        dispatch_narrow(p, [&](auto w) {
            launch_gemm_exact_list<decltype(w)::value>(A, B, C, n, l, p, st, s, list, count);
        });
    }
    {
        Prof pr(MP_K_SPLIT_AUX, 0.0, s);
        dispatch_narrow(p, [&](auto w) {
            launch_gemm_exact<decltype(w)::value>(A, B, C, m, l, n, p, st, s, wa, wb);
        });
    }
    ws.reset(mk);
    return launch_status();
}

// C := A B for (possibly strided) views, with the recursion's buffers carved
// from ws (which must hold gemm_ws_bytes(...)).  Stream-ordered.
size_t gemm_ws_bytes(int algo, int64_t m, int64_t l, int64_t n, int cutoff, int policy, int L)
{
    if (algo == MP_SPLIT) return (m > 0 && l > 0 && n > 0) ? split_ws_bytes(m, l, n, 64 * L) : 0;
    if (algo != MP_STRASSEN && algo != MP_WINOGRAD) return 0;
    if (m <= 0 || l <= 0 || n <= 0) return 0;
    auto lv = plan(m, l, n, cutoff, policy);
    return lv.size() <= 1 ? 0 : recursion_bytes(lv, L);
}

int gemm_core(int algo, int cutoff, int policy, int64_t m, int64_t l, int64_t n, int p, BMat A,
              BMat B, BMat C, Workspace &ws, DevStatus *st, cudaStream_t s)
{
    if (m == 0 || n == 0) return MP_OK;
    const int L = limbs_of(p);
    if (l == 0) {
        Prof pr(MP_K_ELEMENTWISE, (double)m * n, s);
        fill_zero_kernel<<<(unsigned)std::min<int64_t>((m * n + 127) / 128, 152 * 32), 128, 0, s>>>(
            C, m, n, L);
        return launch_status();
    }
    if (algo == MP_SIMPLE) {
        Prof pr(MP_K_SIMPLE, (double)m * l * n, s);
        dispatch(p, [&](auto w) {
            launch_gemm_simple<decltype(w)::value>(A, B, C, m, l, n, p, st, s);
        });
        return launch_status();
    }
    if ((algo == MP_SPLIT || algo == MP_EXACT) && p > MP_PREC_EXACT_MAX) return MP_ERR_UNSUPPORTED;
    if (algo == MP_SPLIT) {
        return run_split(m, l, n, p, A, B, C, ws, st, s);
    }
    if (algo == MP_EXACT) {
        Prof pr(MP_K_EXACT, (double)m * l * n, s);
        dispatch_narrow(p, [&](auto w) {
            launch_gemm_exact<decltype(w)::value>(A, B, C, m, l, n, p, st, s);
        });
        return launch_status();
    }
    auto lv = plan(m, l, n, cutoff, policy);
    if (algo == MP_BLOCK || lv.size() <= 1) {
        Prof pr(MP_K_LEAF, (double)m * l * n, s);
        dispatch(p, [&](auto w) {
            if (launch_gemm_block<decltype(w)::value>(A, B, C, 1, m, l, n, p, st, s, g_ts.leaf_tma))
                pr.reclass(MP_K_LEAF_TMA);
        });
        return launch_status();
    }
    int rc = MP_OK;
    const size_t mk = ws.mark();
    dispatch(p, [&](auto w) {
        rc = run_recursion<decltype(w)::value>(algo, lv, p, A, B, C, ws, st, s);
    });
    ws.reset(mk);
    return rc;
}

BMat sub_view(BMat M, int64_t r0, int64_t c0)
{
    BMat v = M;
    v.limb += r0 * M.ld + c0;
    v.exp += r0 * M.ld + c0;
    v.sign += r0 * M.ld + c0;
    return v;
}

}  // namespace

static size_t lu_ws_bytes(int64_t n, int p, int panel, int algo, int cutoff, int policy)
{
    const int L = limbs_of(p);
    const int64_t K = std::min<int64_t>(panel, n);
    const int64_t nt = n - K;                              // largest trailing block
    size_t b = mat_bytes(1, nt, nt, L) + mat_bytes(1, n, 1, L) + padded((size_t)n * 8);
    b += padded((size_t)mpg::LU_COL_MAX_CTAS * 8) + padded(sizeof(unsigned));
    b += gemm_ws_bytes(algo, nt, K, nt, cutoff, policy, L) + 512;
    return b;
}

namespace mpg {
int auto_cutoff(int p);
int resolve_cutoff(int cutoff, int p);

// C := A B with the recursion's buffers carved from a caller-supplied device
// block [base, base + bytes); nothing is allocated.  Returns MP_ERR_NOMEM if
// the block is too small.  Used by the static-scratch entry point.
int gemm_in_block(int algo, int cutoff, int policy, int64_t m, int64_t l, int64_t n, int p,
                  const mpmat_t *A, const mpmat_t *B, mpmat_t *C, void *base, size_t bytes,
                  DevStatus *st, cudaStream_t s)
{
    const size_t need = gemm_ws_bytes(algo, m, l, n, cutoff, policy, limbs_of(p));
    if (need > bytes) return MP_ERR_NOMEM;
    Workspace ws;
    ws.base = (char *)base;
    ws.size = bytes;
    ws.used = 0;
    ws.s = s;
    return gemm_core(algo, cutoff, policy, m, l, n, p, bmat(A), bmat(B), bmat(C), ws, st, s);
}

size_t gemm_scratch_bytes(int algo, int64_t m, int64_t l, int64_t n, int cutoff, int policy, int p)
{
    return gemm_ws_bytes(algo, m, l, n, cutoff == 0 ? auto_cutoff(p) : cutoff, policy, limbs_of(p));
}

bool gemm_args_ok(int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo, int32_t cutoff,
                  const mpmat_t *A, const mpmat_t *B, const mpmat_t *C)
{
    if (!valid_prec(prec) || m < 0 || l < 0 || n < 0) return false;
    if (algo < MP_SIMPLE || algo > MP_WINOGRAD) return false;
    if ((algo == MP_STRASSEN || algo == MP_WINOGRAD) && cutoff < 0) return false;
    if (!valid_mat(A, m, l, prec) || !valid_mat(B, l, n, prec) || !valid_mat(C, m, n, prec))
        return false;
    return !(overlaps(C, A) || overlaps(C, B));
}

cudaStream_t current_stream() { return g_ts.stream; }

size_t lu_scratch_bytes(int64_t n, int p, int panel, int algo, int cutoff, int policy)
{
    return lu_ws_bytes(n, p, panel, algo, cutoff == 0 ? auto_cutoff(p) : cutoff, policy);
}

// C_b = A_b B_b for a batch of equally shaped products by the Block kernel
// (the server's batched launches).  Stream-ordered.
int gemm_block_batched(int p, BMat A, BMat B, BMat C, int64_t batch, int64_t m, int64_t l,
                       int64_t n, cudaStream_t s)
{
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    Prof pr(MP_K_LEAF, (double)batch * m * l * n, s);
    dispatch(p, [&](auto w) {
        if (launch_gemm_block<decltype(w)::value>(A, B, C, batch, m, l, n, p, st, s, g_ts.leaf_tma))
            pr.reclass(MP_K_LEAF_TMA);
    });
    return launch_status();
}

// Several products C_i := A_i B_i of one precision on stream s (the serving
// loop's groups), each computed exactly as mpgemm computes it with the odd
// policy MP_PEEL: Strassen / Winograd products run their operand sums and
// peel borders, then the leaves of every product in the group go to one
// grouped Block launch (Simple and Block products, and recursions of depth
// 0, as a single leaf of their own shape: Simple and Block give the same
// bits), then each product's combinations and fix-ups.  it[i].ws holds
// gemm_scratch_bytes(...) bytes of device memory for product i.
int gemm_group(GroupGemm *it, int count, int p, cudaStream_t s)
{
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    dispatch(p, [&](auto w) {
        constexpr int WW = decltype(w)::value;
        const int L = limbs_of(p);
        std::vector<RecState> rs((size_t)count);
        std::vector<char> rec((size_t)count, 0);
        LeafGroup grp;
        grp.count = 0;
        double units = 0;
        auto flush = [&]() {
            if (!grp.count) return;
            Prof pr(MP_K_LEAF, units, s);
            launch_gemm_block_group<WW>(grp, p, st, s);
            grp.count = 0;
            units = 0;
        };
        for (int i = 0; i < count; ++i) {
            GroupGemm &g = it[i];
            if (g.m == 0 || g.n == 0) continue;
            if (g.l == 0) {
                Prof pr(MP_K_ELEMENTWISE, (double)g.m * g.n, s);
                fill_zero_kernel<<<(unsigned)std::min<int64_t>((g.m * g.n + 127) / 128, 152 * 32), 128, 0, s>>>(
                    g.C, g.m, g.n, L);
                continue;
            }
            LeafBatch lb;
            const int cutoff = resolve_cutoff(g.cutoff, p);
            auto lv = plan(g.m, g.l, g.n, cutoff, MP_PEEL);
            if ((g.algo == MP_STRASSEN || g.algo == MP_WINOGRAD) && lv.size() > 1) {
                Workspace ws;
                ws.base = (char *)g.ws;
                ws.size = g.ws_bytes;
                ws.used = 0;
                ws.s = s;
                rec_down<WW>(rs[i], g.algo, lv, p, g.A, g.B, g.C, ws, s);
                if (rec_has_borders<WW>(rs[i])) rec_borders<WW>(rs[i], p, st, s);
                rec[i] = 1;
                const int D = (int)lv.size() - 1;
                lb = LeafBatch{rs[i].A[D], rs[i].B[D], rs[i].C[D], rs[i].leaves, lv[D].m, lv[D].l, lv[D].n, 0, 0};
            } else {
                lb = LeafBatch{g.A, g.B, g.C, 1, g.m, g.l, g.n, 0, 0};
            }
            units += (double)lb.batch * lb.m * lb.l * lb.n;
            grp.batch[grp.count++] = lb;
            if (grp.count == LEAF_GROUP_MAX) flush();
        }
        flush();
        for (int i = 0; i < count; ++i)
            if (rec[i]) rec_up<WW>(rs[i], p, st, s);
    });
    return launch_status();
}

// +0 in every element of a batch of rows x cols matrices
int fill_zero_batched(BMat M, int64_t batch, int64_t rows, int64_t cols, int p, cudaStream_t s)
{
    const int L = limbs_of(p);
    for (int64_t b = 0; b < batch; ++b) {
        BMat v = M;
        v.limb += b * M.bs_limb;
        v.exp += b * M.bs_es;
        v.sign += b * M.bs_es;
        fill_zero_kernel<<<(unsigned)std::min<int64_t>((rows * cols + 127) / 128, 152 * 32), 128, 0,
                           s>>>(v, rows, cols, L);
    }
    return launch_status();
}
int current_odd_policy() { return g_ts.odd_policy; }

// Strassen/Winograd cutoff for cutoff = 0: the value that was fastest for
// Winograd on GB300 at n = 1024 and 2048 with cutoffs 16..256 (64 up to 1024
// bits, 32 at 2048 bits, where a leaf product costs most against the
// additions; the wide class takes 32 as well).  Leaves narrower than the
// 32-column tile of the Block kernel waste lanes, so 16 was slowest always.
int auto_cutoff(int p)
{
    return wclass(p) <= 32 ? 64 : 32;
}

int resolve_cutoff(int cutoff, int p)
{
    return cutoff == 0 ? auto_cutoff(p) : cutoff;
}
}  // namespace mpg

// ======================================================================= ABI
extern "C" {

int mp_version(void) { return 100; }

int mp_set_stream(void *stream)
{
    g_ts.stream = (cudaStream_t)stream;
    return MP_OK;
}

int mp_set_workspace(void *ptr, size_t bytes)
{
    g_ts.ws = ptr;
    g_ts.ws_bytes = ptr ? bytes : 0;
    return MP_OK;
}

int mp_set_odd_policy(int policy)
{
    if (policy != MP_PEEL && policy != MP_MIXED) return MP_ERR_ARG;
    g_ts.odd_policy = policy;
    return MP_OK;
}

int mp_set_lu(int panel, int algo, int cutoff)
{
    if (panel < 1 || algo < MP_SIMPLE || algo > MP_WINOGRAD || cutoff < 0) return MP_ERR_ARG;
    g_ts.lu_panel = panel;
    g_ts.lu_algo = algo;
    g_ts.lu_cutoff = cutoff;
    return MP_OK;
}

int mp_set_lu_pivoting(int on)
{
    if (on != 0 && on != 1) return MP_ERR_ARG;
    g_ts.lu_pivoting = on == 1;
    return MP_OK;
}

const char *mp_strerror(int status)
{
    switch (status) {
    case MP_OK: return "ok";
    case MP_ERR_ARG: return "invalid argument";
    case MP_ERR_NOMEM: return "workspace allocation failed";
    case MP_ERR_SINGULAR: return "zero pivot: matrix is singular";
    case MP_ERR_TIMEOUT: return "device wait timed out";
    case MP_ERR_CUDA: return "CUDA runtime error";
    case MP_ERR_RANGE: return "exponent out of range";
    case MP_ERR_UNSUPPORTED: return "unsupported (e.g. exponent spread too wide for exact accumulation)";
    case MP_ERR_SCRATCH: return "product needs more than the static scratch array holds";
    default: return "unknown status";
    }
}

int mp_sync_status(void)
{
    cudaError_t e = cudaStreamSynchronize(g_ts.stream);
    if (e != cudaSuccess) return MP_ERR_CUDA;
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    DevStatus h{};
    if (cudaMemcpy(&h, st, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return MP_ERR_CUDA;
    if (h.flags || h.split_fallbacks) {
        DevStatus init{0u, 0u, INT64_MAX, 0ull};
        cudaMemcpy(st, &init, sizeof init, cudaMemcpyHostToDevice);
    }
    // conditions recorded by mpgemm_noalloc in its own static status word
    h.flags |= noalloc_take_flags();
    g_ts.split_fallbacks = (long long)h.split_fallbacks;
    g_ts.singular_col = (h.singular_col == INT64_MAX) ? -1 : h.singular_col;
    if (h.flags & ST_TIMEOUT) return MP_ERR_TIMEOUT;
    if (h.flags & ST_SINGULAR) return MP_ERR_SINGULAR;
    if (h.flags & ST_DIVZERO) return MP_ERR_ARG;
    if (h.flags & ST_RANGE) return MP_ERR_RANGE;
    if (h.flags & ST_WIDE) return MP_ERR_UNSUPPORTED;
    return MP_OK;
}

int mp_wait_selftest(int64_t cycles)
{
    if (cycles < 1 || cycles > ((int64_t)1 << 32)) return MP_ERR_ARG;
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    launch_wait_selftest(st, (long long)cycles, g_ts.stream);
    const int rc = launch_status();
    if (rc != MP_OK) return rc;
    return mp_sync_status();
}

int64_t mp_singular_column(void) { return g_ts.singular_col; }

int64_t mp_split_fallbacks(void) { return g_ts.split_fallbacks; }

int mp_set_split_truncation(int on)
{
    if (on != 0 && on != 1) return MP_ERR_ARG;
    g_ts.split_truncate = on == 1;
    return MP_OK;
}

int mp_set_leaf_tma(int on)
{
    if (on != 0 && on != 1) return MP_ERR_ARG;
    g_ts.leaf_tma = on == 1;
    return MP_OK;
}

int mp_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.drain();
    g_prof.on = on != 0;
    if (g_prof.on) {
        for (int i = 0; i < MP_K_COUNT; ++i) {
            g_prof.launches[i] = 0;
            g_prof.ms[i] = 0.0;
            g_prof.units[i] = 0.0;
        }
    }
    return MP_OK;
}

int mp_profile_read(int cls, int64_t *launches, double *ms, double *units)
{
    if (cls < 0 || cls >= MP_K_COUNT) return MP_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.drain();
    if (launches) *launches = g_prof.launches[cls];
    if (ms) *ms = g_prof.ms[cls];
    if (units) *units = g_prof.units[cls];
    return MP_OK;
}

int mp_elementwise(int op, const mpmat_t *X, const mpmat_t *Y, mpmat_t *R)
{
    if (op < 0 || op > 7 || !X || !Y || !R) return MP_ERR_ARG;
    const int p = X->prec;
    if (!valid_prec(p)) return MP_ERR_ARG;
    if (op >= 4 && wclass(p) > 32) return MP_ERR_UNSUPPORTED;
    const int64_t rows = X->rows, cols = X->cols;
    if (!valid_mat(X, rows, cols, p) || !valid_mat(Y, rows, cols, p) || !valid_mat(R, rows, cols, p))
        return MP_ERR_ARG;
    // R may alias an input only exactly
    auto same = [](const mpmat_t *a, const mpmat_t *b) {
        return a->limb == b->limb && a->exp == b->exp && a->sign == b->sign && a->ld == b->ld &&
               a->plane == b->plane;
    };
    if ((overlaps(R, X) && !same(R, X)) || (overlaps(R, Y) && !same(R, Y))) return MP_ERR_ARG;
    if (rows == 0 || cols == 0) return MP_OK;
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    Prof pr(MP_K_ELEMENTWISE, (double)rows * cols, g_ts.stream);
    dispatch(p, [&](auto w) {
        constexpr int WW = decltype(w)::value;
        if (op < 4) {
            launch_elementwise<WW>(op, bmat(X), bmat(Y), bmat(R), rows, cols, p, st, g_ts.stream);
        } else if constexpr (WW <= 32) {
            launch_elementwise_warp<WW>(op - 4, bmat(X), bmat(Y), bmat(R), rows, cols, p, st, g_ts.stream);
        }
    });
    return launch_status();
}

int mp_convert(const mpmat_t *X, mpmat_t *R)
{
    if (!X || !R || !valid_prec(X->prec) || !valid_prec(R->prec)) return MP_ERR_ARG;
    const int64_t rows = X->rows, cols = X->cols;
    if (!valid_mat(X, rows, cols, X->prec) || !valid_mat(R, rows, cols, R->prec)) return MP_ERR_ARG;
    if (overlaps(X, R)) return MP_ERR_ARG;
    if (rows == 0 || cols == 0) return MP_OK;
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    const int pmax = std::max(X->prec, R->prec);
    Prof pr(MP_K_ELEMENTWISE, (double)rows * cols, g_ts.stream);
    dispatch(pmax, [&](auto w) {
        launch_convert<decltype(w)::value>(bmat(X), X->prec, bmat(R), R->prec, rows, cols, st,
                                           g_ts.stream);
    });
    return launch_status();
}

size_t mpgemm_workspace_size(int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo,
                             int32_t cutoff)
{
    if (algo == MP_SPLIT)
        return (m > 0 && l > 0 && n > 0 && valid_prec(prec)) ? split_ws_bytes(m, l, n, prec) : 0;
    if (algo != MP_STRASSEN && algo != MP_WINOGRAD) return 0;
    if (cutoff < 0 || m <= 0 || l <= 0 || n <= 0 || !valid_prec(prec)) return 0;
    cutoff = resolve_cutoff(cutoff, prec);
    auto lv = plan(m, l, n, cutoff, g_ts.odd_policy);
    if (lv.size() <= 1) return 0;
    return recursion_bytes(lv, limbs_of(prec));
}

int mpgemm(int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo, int32_t cutoff,
           const mpmat_t *A, const mpmat_t *B, mpmat_t *C)
{
    if (!valid_prec(prec) || m < 0 || l < 0 || n < 0) return MP_ERR_ARG;
    if (algo < MP_SIMPLE || algo > MP_SPLIT) return MP_ERR_ARG;
    if ((algo == MP_STRASSEN || algo == MP_WINOGRAD) && cutoff < 0) return MP_ERR_ARG;
    cutoff = resolve_cutoff(cutoff, prec);
    if (!valid_mat(A, m, l, prec) || !valid_mat(B, l, n, prec) || !valid_mat(C, m, n, prec))
        return MP_ERR_ARG;
    if (overlaps(C, A) || overlaps(C, B)) return MP_ERR_ARG;
    if (m == 0 || n == 0) return MP_OK;
    cudaStream_t s = g_ts.stream;
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    Workspace ws;
    int rc = ws.acquire(gemm_ws_bytes(algo, m, l, n, cutoff, g_ts.odd_policy, limbs_of(prec)), s);
    if (rc != MP_OK) return rc;
    return gemm_core(algo, cutoff, g_ts.odd_policy, m, l, n, prec, bmat(A), bmat(B), bmat(C), ws,
                     st, s);
}


int mpgemm_batched(int64_t batch, int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo,
                   const mpmat_t *A, const mpmat_t *B, mpmat_t *C)
{
    if (!valid_prec(prec) || batch < 0 || m < 0 || l < 0 || n < 0) return MP_ERR_ARG;
    if (algo != MP_SIMPLE && algo != MP_BLOCK)
        return (algo >= MP_STRASSEN && algo <= MP_SPLIT) ? MP_ERR_UNSUPPORTED : MP_ERR_ARG;
    if (!valid_mat(A, batch * m, l, prec) || !valid_mat(B, batch * l, n, prec) ||
        !valid_mat(C, batch * m, n, prec))
        return MP_ERR_ARG;
    if (overlaps(C, A) || overlaps(C, B)) return MP_ERR_ARG;
    if (batch == 0 || m == 0 || n == 0) return MP_OK;
    cudaStream_t s = g_ts.stream;
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    const int L = limbs_of(prec);
    if (l == 0) {
        Prof pr(MP_K_ELEMENTWISE, (double)batch * m * n, s);
        fill_zero_kernel<<<(unsigned)std::min<int64_t>((batch * m * n + 127) / 128, 152 * 32), 128, 0,
                           s>>>(bmat(C), batch * m, n, L);
        return launch_status();
    }
    BMat a = bmat(A), b = bmat(B), c = bmat(C);
    a.bs_limb = a.bs_es = m * A->ld;
    b.bs_limb = b.bs_es = l * B->ld;
    c.bs_limb = c.bs_es = m * C->ld;
    Prof pr(MP_K_LEAF, (double)batch * m * l * n, s);
    dispatch(prec, [&](auto w) {
        if (launch_gemm_block<decltype(w)::value>(a, b, c, batch, m, l, n, prec, st, s, g_ts.leaf_tma))
            pr.reclass(MP_K_LEAF_TMA);
    });
    return launch_status();
}

size_t mplu_workspace_size(int64_t n, int32_t prec)
{
    if (n <= 0 || !valid_prec(prec)) return 0;
    return lu_ws_bytes(n, prec, g_ts.lu_panel, g_ts.lu_algo, resolve_cutoff(g_ts.lu_cutoff, prec),
                       g_ts.odd_policy);
}

int mplu(int64_t n, int32_t prec, mpmat_t *A, int64_t *piv, const mpmat_t *b, mpmat_t *x)
{
    if (!valid_prec(prec) || n < 0 || !valid_mat(A, n, n, prec)) return MP_ERR_ARG;
    if (n > 0 && !piv) return MP_ERR_ARG;
    if (x) {
        if (!b || !valid_mat(b, n, 1, prec) || !valid_mat(x, n, 1, prec)) return MP_ERR_ARG;
        if (overlaps(x, A) || overlaps(x, b) || overlaps(b, A)) return MP_ERR_ARG;
    }
    if (n == 0) return MP_OK;
    cudaStream_t s = g_ts.stream;
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    const int K = g_ts.lu_panel, algo = g_ts.lu_algo, cutoff = resolve_cutoff(g_ts.lu_cutoff, prec);
    const int policy = g_ts.odd_policy;
    const bool pivoting = g_ts.lu_pivoting;
    const int L = limbs_of(prec);
    Workspace ws;
    int rc = ws.acquire(lu_ws_bytes(n, prec, K, algo, cutoff, policy), s);
    if (rc != MP_OK) return rc;
    const int64_t nt0 = n - std::min<int64_t>(K, n);
    BMat T = carve(ws, 1, nt0, nt0, L);                    // trailing product, ld = nt0
    BMat y = carve(ws, 1, n, 1, L);
    int64_t *perm = (int64_t *)ws.take((size_t)n * 8);
    int64_t *cand = (int64_t *)ws.take((size_t)mpg::LU_COL_MAX_CTAS * 8);
    unsigned *ticket = (unsigned *)ws.take(sizeof(unsigned));
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned), s) != cudaSuccess) return MP_ERR_CUDA;
    const BMat A0 = bmat(A);
    dispatch(prec, [&](auto w) {
        constexpr int WW = decltype(w)::value;
        const bool fused = lu_fused_ok<WW>(K);
        for (int64_t j0 = 0; j0 < n && rc == MP_OK; j0 += K) {
            const int64_t je = std::min<int64_t>(j0 + K, n);
            {
                if (fused) {
                    // The panel in sub-panels of lu_sub_width<W>() columns.  A sub-panel
                    // [c0, c1) first takes the updates of the panel's earlier
                    // columns k in [j0, c0) on its own columns from row c0
                    // down (subtracting Block product, k ascending), then is
                    // factored column by column over its own columns only,
                    // so that all rows below the current column stay in one
                    // state and the row exchanges move consistent rows.
                    // Afterwards its rows take their updates on the panel's
                    // later columns: k in [j0, c0) by the subtracting Block
                    // product, then k in [c0, c1) by the triangular solve.
                    // Every element receives a_ij = RN(a_ij - RN(l_ik u_kj))
                    // for the same k in the same order as in the
                    // right-looking panel, and each latency-bound column step
                    // is one multiply-add deep.  Row exchanges: the panel's
                    // columns at once, the rest after the panel.
                    {
                        Prof pr(MP_K_LU, (double)(n - j0), s);
                        launch_lu_pivot<WW>(A0, n, j0, piv, prec, st, s, j0, je, pivoting);
                    }
                    constexpr int64_t SW = lu_sub_width<WW>();
                    for (int64_t c0 = j0; c0 < je; c0 += SW) {
                        const int64_t c1 = std::min<int64_t>(c0 + SW, je);
                        if (c0 > j0) {
                            {
                                Prof pr(MP_K_LU_UPDATE, (double)(n - c0) * (c0 - j0) * (c1 - c0), s);
                                launch_gemm_sub<WW>(sub_view(A0, c0, j0), sub_view(A0, j0, c0), sub_view(A0, c0, c0),
                                                    n - c0, c0 - j0, c1 - c0, prec, st, s);
                            }
                            Prof pr(MP_K_LU, (double)(n - c0), s);
                            launch_lu_pivot<WW>(A0, n, c0, piv, prec, st, s, j0, je, pivoting);
                        }
                        for (int64_t k = c0; k < c1; ++k) {
                            Prof pr(MP_K_LU, (double)(c1 - k) * (n - k), s);
                            launch_lu_column<WW>(A0, n, j0, k, je, c1, piv, prec, st, cand, ticket, s, pivoting);
                        }
                        if (c1 < je) {
                            if (c0 > j0) {
                                Prof pr(MP_K_LU_UPDATE, (double)(c1 - c0) * (c0 - j0) * (je - c1), s);
                                launch_gemm_sub<WW>(sub_view(A0, c0, j0), sub_view(A0, j0, c1), sub_view(A0, c0, c1),
                                                    c1 - c0, c0 - j0, je - c1, prec, st, s);
                            }
                            Prof pr(MP_K_LU_TRSM, (double)(c1 - c0) * (c1 - c0 - 1) / 2 * (je - c1), s);
                            launch_lu_u12<WW>(A0, je, c0, c1, prec, st, s);
                        }
                    }
                    Prof pr(MP_K_LU, (double)(n - (je - j0)), s);
                    launch_lu_laswp<WW>(A0, n, j0, je, piv, prec, s);
                } else {
                    Prof pr(MP_K_LU, (double)(je - j0) * (n - j0), s);
                    for (int64_t k = j0; k < je; ++k) {
                        launch_lu_pivot<WW>(A0, n, k, piv, prec, st, s, 0, n, pivoting);
                        launch_lu_divide<WW>(A0, n, k, prec, s);
                        launch_lu_rank1<WW>(A0, k, k + 1, n, k + 1, je, prec, st, s);
                    }
                }
            }
            if (je >= n) break;
            {
                Prof pr(MP_K_LU_TRSM, (double)(je - j0) * (je - j0 - 1) / 2 * (n - je), s);
                if (fused)                                     // U12 = L11^-1 A12
                    launch_lu_u12<WW>(A0, n, j0, je, prec, st, s);
                else
                    for (int64_t r = j0; r + 1 < je; ++r)
                        launch_lu_rank1<WW>(A0, r, r + 1, je, je, n, prec, st, s);
            }
            const int64_t nt = n - je;
            BMat Tv = T;
            Tv.ld = nt;
            Tv.plane = nt * nt;
            rc = gemm_core(algo, cutoff, policy, nt, je - j0, nt, prec, sub_view(A0, je, j0),
                           sub_view(A0, j0, je), Tv, ws, st, s);
            {
                Prof pr(MP_K_LU_UPDATE, (double)nt * nt, s);
                const BMat A22 = sub_view(A0, je, je);
                launch_elementwise<WW>(1, A22, Tv, A22, nt, nt, prec, st, s);
            }
        }
        if (rc == MP_OK && x) {
            Prof pr(MP_K_LU_SOLVE, (double)n * n, s);
            launch_lu_solve<WW>(A0, n, piv, bmat(b), y, bmat(x), perm, prec, st, s);
        }
    });
    if (rc != MP_OK) return rc;
    return launch_status();
}

int mplu_solve(int64_t n, int32_t prec, const mpmat_t *LU, const int64_t *piv, const mpmat_t *B, mpmat_t *X)
{
    if (!valid_prec(prec) || n < 0 || !valid_mat(LU, n, n, prec) || !B || !X) return MP_ERR_ARG;
    const int64_t nrhs = B->cols;
    if (!valid_mat(B, n, nrhs, prec) || !valid_mat(X, n, nrhs, prec)) return MP_ERR_ARG;
    if (n > 0 && nrhs > 0 && !piv) return MP_ERR_ARG;
    if (overlaps(X, LU) || overlaps(X, B)) return MP_ERR_ARG;
    if (n == 0 || nrhs == 0) return MP_OK;
    cudaStream_t s = g_ts.stream;
    DevStatus *st = status_ptr();
    if (!st) return MP_ERR_CUDA;
    const int L = limbs_of(prec);
    Workspace ws;
    int rc = ws.acquire(mat_bytes(1, n, nrhs, L) + padded((size_t)n * 8) + 512, s);
    if (rc != MP_OK) return rc;
    BMat Y = carve(ws, 1, n, nrhs, L);
    int64_t *perm = (int64_t *)ws.take((size_t)n * 8);
    Prof pr(MP_K_LU_SOLVE, (double)n * n * nrhs, s);
    dispatch(prec, [&](auto w) {
        launch_lu_solve_multi<decltype(w)::value>(bmat(LU), n, piv, bmat(B), Y, bmat(X), nrhs, perm, prec, st, s);
    });
    return launch_status();
}

}  // extern "C"

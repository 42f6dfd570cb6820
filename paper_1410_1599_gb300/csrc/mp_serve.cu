// mp_serve.cu -- continuous batching of MP GEMM and LU-solve requests
// (the serving loop of include/mpgemm.h).
//
// One scheduler thread per server owns the device work: it admits queued
// requests in arrival order while their device memory fits the budget and a
// slot (a CUDA stream) is free, looking past a request that does not fit
// yet (bounded look-ahead) so that small requests keep flowing; it groups
// queued Simple/Block GEMMs of one precision and size bucket into a single
// grouped Block launch, and other GEMMs of one precision and size class into
// leaf groups (each request's own recursion, the leaves of all of them in
// shared grouped launches); and it retires finished work by polling events.
// Operands, results and factors stay in device memory from admission to
// retirement; memory is taken and returned stream-ordered.
//
// Repeated request shapes run from captured CUDA graphs: the second time a
// single request's signature (kind, sizes, precision, algorithm, cutoff,
// panel) is seen, its device work is captured once into a graph over
// buffers the cache owns; later requests with that signature copy their
// operands into those buffers, launch the graph and copy the result out.
// Cached buffers count against the memory budget and idle entries are
// evicted (least recently used) when a request needs the room.
#include <algorithm>
#include <map>
#include <tuple>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mpgemm.h"
#include "mp_internal.h"

namespace mpg {
int gemm_block_batched(int p, BMat A, BMat B, BMat C, int64_t batch, int64_t m, int64_t l,
                       int64_t n, cudaStream_t s);
int fill_zero_batched(BMat M, int64_t batch, int64_t rows, int64_t cols, int p, cudaStream_t s);
size_t gemm_scratch_bytes(int algo, int64_t m, int64_t l, int64_t n, int cutoff, int policy, int p);
size_t lu_scratch_bytes(int64_t n, int p, int panel, int algo, int cutoff, int policy);
int gemm_group(GroupGemm *it, int count, int p, cudaStream_t s);
}  // namespace mpg

using namespace mpg;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kLookAhead = 32;     // queued requests scanned past a blocked head
constexpr int kMaxBatch = 64;      // requests per grouped launch
constexpr int kMaxGroup = 8;       // GEMMs per leaf group
const int64_t kBuckets[] = {64, 128, 256, 512};
const int64_t kClasses[] = {256, 512, 1024, 2048};

int limbs(int p) { return (p + 63) / 64; }
size_t elem_bytes(int p) { return (size_t)8 * limbs(p) + 9; }
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Req {
    mp_request_t r;
    Clock::time_point t_submit;
    int state = MP_REQ_PENDING;
    int64_t bucket = 0;           // > 0 if batchable
    size_t bytes = 0;             // device footprint when run alone
};

struct GraphEntry;

struct Unit {                     // admitted work on one slot
    std::vector<Req *> reqs;
    bool group = false;           // GEMMs of one precision sharing their leaf launches
    GraphEntry *graph = nullptr;  // cached graph the unit ran from (busy until retired)
    int slot = -1;
    cudaEvent_t done = nullptr;
    size_t bytes = 0;
    int rc = MP_OK;
};

struct Finished {
    int64_t id;
    int32_t status;
    double ms;
};

typedef std::tuple<int32_t, int32_t, int64_t, int64_t, int64_t, int32_t, int32_t, int32_t> Sig;

Sig signature(const mp_request_t &r)
{
    const bool lu = r.kind == MP_REQ_LU_SOLVE;
    return Sig(r.kind, r.prec, r.m, lu ? 0 : r.l, lu ? 0 : r.n, r.algo, r.cutoff,
               lu ? (r.lu_panel > 0 ? r.lu_panel : 128) : 0);
}

struct GraphEntry {
    Sig sig;
    cudaGraphExec_t exec = nullptr;
    char *mem = nullptr;
    size_t bytes = 0;
    mpmat_t A{}, B{}, C{};        // GEMM: A, B, C; LU solve: A, b, x
    int64_t *piv = nullptr;
    bool busy = false;
    uint64_t last = 0;
};

// size class of a GEMM for leaf groups: the bound on its largest dimension
// (0: too large, or not a GEMM)
int64_t group_class(const mp_request_t &r)
{
    if (r.kind != MP_REQ_GEMM) return 0;
    const int64_t mx = std::max(r.m, std::max(r.l, r.n));
    for (int64_t c : kClasses)
        if (mx <= c) return c;
    return 0;
}

bool batchable(const mp_request_t &r, int64_t *bucket)
{
    if (r.kind != MP_REQ_GEMM || (r.algo != MP_SIMPLE && r.algo != MP_BLOCK)) return false;
    const int64_t mx = std::max(r.m, std::max(r.l, r.n));
    for (int64_t b : kBuckets)
        if (mx <= b) { *bucket = b; return true; }
    return false;
}

}  // namespace

struct mp_server {
    int device = 0;
    size_t budget = 0, used = 0, peak = 0;
    std::vector<cudaStream_t> streams;
    std::vector<bool> busy;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<Req *> queue;
    std::vector<Unit *> running;
    std::vector<Finished> finished;
    std::thread th;
    bool stop = false;
    int64_t n_submitted = 0, n_completed = 0, n_batches = 0, n_batched_reqs = 0;
    int64_t outstanding = 0;
    // graph cache (touched by the scheduler thread only; `used` under mu)
    int graph_slots = 8;
    std::vector<GraphEntry *> graphs;
    std::map<Sig, int> seen;      // signatures seen once (graph-cache candidates), at most kSeenMax
    static constexpr size_t kSeenMax = 1 << 16;
    void mark_seen(const Sig &sig)
    {
        if (seen.size() >= kSeenMax) seen.clear();   // forget old shapes rather than grow without bound
        seen[sig] = 1;
    }
    uint64_t tick = 0;
    int64_t n_captures = 0, n_replays = 0;
    size_t graph_bytes = 0;

    // ------------------------------------------------------------- footprint
    static size_t footprint(const mp_request_t &r)
    {
        const int p = r.prec;
        if (r.kind == MP_REQ_GEMM)
            return mat_size(p, r.m, r.l) + mat_size(p, r.l, r.n) + mat_size(p, r.m, r.n) +
                   gemm_scratch_bytes(r.algo, r.m, r.l, r.n, r.cutoff, MP_PEEL, p);
        const int64_t n = r.m;
        return mat_size(p, n, n) + 2 * mat_size(p, n, 1) + align256((size_t)n * 8) +
               lu_scratch_bytes(n, p, r.lu_panel > 0 ? r.lu_panel : 128, r.algo, r.cutoff, MP_PEEL);
    }

    static size_t batch_bytes(int p, int64_t b, int64_t count)
    {
        return 3 * mat_size(p, count * b, b);
    }

    // ---------------------------------------------------------------- launch
    static void mat_on(mpmat_t &M, int p, int64_t rows, int64_t cols, char *base)
    {
        const size_t e = (size_t)rows * cols;
        M.prec = p;
        M.reserved = 0;
        M.rows = rows;
        M.cols = cols;
        M.ld = cols;
        M.plane = rows * cols;
        M.limb = (uint64_t *)base;
        M.exp = (int64_t *)(base + align256(e * 8 * limbs(p)));
        M.sign = (int8_t *)(base + align256(e * 8 * limbs(p)) + align256(e * 8));
    }
    static size_t mat_size(int p, int64_t rows, int64_t cols)
    {
        const size_t e = (size_t)rows * cols;
        return align256(e * 8 * limbs(p)) + align256(e * 8) + align256(e);
    }
    static int h2d(const mpmat_t &M, const uint64_t *l, const int64_t *e, const int8_t *s,
                   cudaStream_t st)
    {
        const size_t n = (size_t)M.rows * M.cols;
        if (!n) return MP_OK;
        cudaMemcpyAsync(M.limb, l, n * 8 * limbs(M.prec), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(M.exp, e, n * 8, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(M.sign, s, n, cudaMemcpyHostToDevice, st);
        return cudaGetLastError() == cudaSuccess ? MP_OK : MP_ERR_CUDA;
    }
    static int d2h(const mpmat_t &M, uint64_t *l, int64_t *e, int8_t *s, cudaStream_t st)
    {
        const size_t n = (size_t)M.rows * M.cols;
        if (!n) return MP_OK;
        cudaMemcpyAsync(l, M.limb, n * 8 * limbs(M.prec), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(e, M.exp, n * 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(s, M.sign, n, cudaMemcpyDeviceToHost, st);
        return cudaGetLastError() == cudaSuccess ? MP_OK : MP_ERR_CUDA;
    }

    // ----------------------------------------------------------- graph cache
    // device buffers of one cached signature: the request's operands and
    // result (plus the pivot vector of an LU solve)
    static size_t entry_bytes(const mp_request_t &r)
    {
        const int p = r.prec;
        if (r.kind == MP_REQ_GEMM) return mat_size(p, r.m, r.l) + mat_size(p, r.l, r.n) + mat_size(p, r.m, r.n);
        return mat_size(p, r.m, r.m) + 2 * mat_size(p, r.m, 1) + align256((size_t)r.m * 8);
    }

    // release an idle entry (scheduler thread, mu held)
    void evict_locked(GraphEntry *g)
    {
        graphs.erase(std::find(graphs.begin(), graphs.end(), g));
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->mem) cudaFree(g->mem);
        cudaDeviceGraphMemTrim(device);           // return the graph's pool memory
        used -= g->bytes;
        graph_bytes -= g->bytes;
        delete g;
    }

    GraphEntry *lru_idle_locked()
    {
        GraphEntry *best = nullptr;
        for (GraphEntry *g : graphs)
            if (!g->busy && (!best || g->last < best->last)) best = g;
        return best;
    }

    // Capture the device work of r over new cache-owned buffers (scheduler
    // thread, mu not held).  nullptr if capture is not possible.
    GraphEntry *capture(const mp_request_t &r, cudaStream_t st)
    {
        GraphEntry *g = new GraphEntry;
        g->sig = signature(r);
        g->bytes = footprint(r);
        if (cudaMalloc((void **)&g->mem, entry_bytes(r)) != cudaSuccess) {
            cudaGetLastError();
            delete g;
            return nullptr;
        }
        const int p = r.prec;
        mp_set_stream(st);
        mp_set_workspace(nullptr, 0);
        mp_set_odd_policy(MP_PEEL);
        if (r.kind == MP_REQ_GEMM) {
            mat_on(g->A, p, r.m, r.l, g->mem);
            mat_on(g->B, p, r.l, r.n, g->mem + mat_size(p, r.m, r.l));
            mat_on(g->C, p, r.m, r.n, g->mem + mat_size(p, r.m, r.l) + mat_size(p, r.l, r.n));
        } else {
            const int64_t n = r.m;
            const size_t sa = mat_size(p, n, n), sv = mat_size(p, n, 1);
            mat_on(g->A, p, n, n, g->mem);
            mat_on(g->B, p, n, 1, g->mem + sa);
            mat_on(g->C, p, n, 1, g->mem + sa + sv);
            g->piv = (int64_t *)(g->mem + sa + 2 * sv);
            mp_set_lu(r.lu_panel > 0 ? r.lu_panel : 128, r.algo, r.cutoff);
        }
        cudaGraph_t graph = nullptr;
        int rc = MP_ERR_CUDA;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            rc = (r.kind == MP_REQ_GEMM)
                     ? mpgemm(r.m, r.l, r.n, p, r.algo, r.cutoff, &g->A, &g->B, &g->C)
                     : mplu(r.m, p, &g->A, g->piv, &g->B, &g->C);
            if (cudaStreamEndCapture(st, &graph) != cudaSuccess) rc = MP_ERR_CUDA;
        }
        if (rc == MP_OK && graph && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) rc = MP_ERR_CUDA;
        if (graph) cudaGraphDestroy(graph);
        if (rc != MP_OK || !g->exec) {
            cudaGetLastError();
            cudaFree(g->mem);
            delete g;
            return nullptr;
        }
        return g;
    }

    // one request through a cached graph
    int run_graph(GraphEntry *g, Req *q, cudaStream_t st)
    {
        const mp_request_t &r = q->r;
        int rc = h2d(g->A, r.a_limb, r.a_exp, r.a_sign, st);
        if (rc == MP_OK) rc = h2d(g->B, r.b_limb, r.b_exp, r.b_sign, st);
        if (rc == MP_OK && cudaGraphLaunch(g->exec, st) != cudaSuccess) rc = MP_ERR_CUDA;
        if (rc == MP_OK) rc = d2h(g->C, r.c_limb, r.c_exp, r.c_sign, st);
        return rc;
    }

    // Run a single request: from the graph cache when its signature is cached
    // (or seen before and there is room to capture it), else directly.
    // Scheduler thread, mu not held; the cache is the scheduler's own.
    int run_request(Unit *u, cudaStream_t st)
    {
        Req *q = u->reqs[0];
        if (graph_slots <= 0) return run_single(q, st);
        const Sig sig = signature(q->r);
        GraphEntry *g = nullptr;
        for (GraphEntry *e : graphs)
            if (e->sig == sig) { g = e; break; }
        if (g && g->busy) return run_single(q, st);     // one entry per signature
        if (!g) {
            if (!seen.count(sig)) {                                 // first sighting
                mark_seen(sig);
                return run_single(q, st);
            }
            // the cache holds the operand buffers and, in the graph's memory
            // pool, the captured work's temporaries: the whole footprint
            const size_t need = footprint(q->r);
            if (need > budget / 16) return run_single(q, st);      // keep the cache small
            {
                std::lock_guard<std::mutex> lk(mu);
                while ((int)graphs.size() >= graph_slots || used + need > budget) {
                    GraphEntry *v = lru_idle_locked();
                    if (!v) break;
                    evict_locked(v);
                }
                if ((int)graphs.size() >= graph_slots || used + need > budget) return run_single(q, st);
                used += need;                      // reserved for the new entry
                graph_bytes += need;
                peak = std::max(peak, used);
            }
            g = capture(q->r, st);
            std::lock_guard<std::mutex> lk(mu);
            if (!g) {
                used -= need;
                graph_bytes -= need;
            } else {
                graphs.push_back(g);
                ++n_captures;
            }
            if (!g) return run_single(q, st);
        }
        g->busy = true;
        g->last = ++tick;
        u->graph = g;
        ++n_replays;
        return run_graph(g, q, st);
    }

    // one request alone on stream st
    int run_single(Req *q, cudaStream_t st)
    {
        const mp_request_t &r = q->r;
        mp_set_stream(st);
        mp_set_workspace(nullptr, 0);
        mp_set_odd_policy(MP_PEEL);
        const int p = r.prec;
        int rc = MP_OK;
        if (r.kind == MP_REQ_GEMM) {
            const size_t sa = mat_size(p, r.m, r.l), sb = mat_size(p, r.l, r.n), sc = mat_size(p, r.m, r.n);
            char *mem = nullptr;
            if (cudaMallocAsync((void **)&mem, sa + sb + sc, st) != cudaSuccess) return MP_ERR_NOMEM;
            mpmat_t A, B, C;
            mat_on(A, p, r.m, r.l, mem);
            mat_on(B, p, r.l, r.n, mem + sa);
            mat_on(C, p, r.m, r.n, mem + sa + sb);
            rc = h2d(A, r.a_limb, r.a_exp, r.a_sign, st);
            if (rc == MP_OK) rc = h2d(B, r.b_limb, r.b_exp, r.b_sign, st);
            if (rc == MP_OK) rc = mpgemm(r.m, r.l, r.n, p, r.algo, r.cutoff, &A, &B, &C);
            if (rc == MP_OK) rc = d2h(C, r.c_limb, r.c_exp, r.c_sign, st);
            cudaFreeAsync(mem, st);
        } else {
            const int64_t n = r.m;
            const size_t sa = mat_size(p, n, n), sv = mat_size(p, n, 1);
            char *mem = nullptr;
            if (cudaMallocAsync((void **)&mem, sa + 2 * sv + align256((size_t)n * 8), st) != cudaSuccess)
                return MP_ERR_NOMEM;
            mpmat_t A, b, x;
            mat_on(A, p, n, n, mem);
            mat_on(b, p, n, 1, mem + sa);
            mat_on(x, p, n, 1, mem + sa + sv);
            int64_t *piv = (int64_t *)(mem + sa + 2 * sv);
            mp_set_lu(r.lu_panel > 0 ? r.lu_panel : 128, r.algo, r.cutoff);
            rc = h2d(A, r.a_limb, r.a_exp, r.a_sign, st);
            if (rc == MP_OK) rc = h2d(b, r.b_limb, r.b_exp, r.b_sign, st);
            if (rc == MP_OK) rc = mplu(n, p, &A, piv, &b, &x);
            if (rc == MP_OK) rc = d2h(x, r.c_limb, r.c_exp, r.c_sign, st);
            cudaFreeAsync(mem, st);
        }
        return rc;
    }

    // Simple/Block GEMMs of one precision and bucket b as one grouped launch
    int run_batch(const std::vector<Req *> &qs, int64_t b, cudaStream_t st)
    {
        const int p = qs[0]->r.prec, L = limbs(p);
        const int64_t k = (int64_t)qs.size();
        const size_t one = mat_size(p, k * b, b);       // k stacked b x b matrices
        char *mem = nullptr;
        if (cudaMallocAsync((void **)&mem, 3 * one, st) != cudaSuccess) return MP_ERR_NOMEM;
        BMat M[3];
        for (int t = 0; t < 3; ++t) {
            mpmat_t v;
            mat_on(v, p, k * b, b, mem + t * one);
            // batch element i: rows [i*b, (i+1)*b) of a (k*b) x b matrix, limb plane k*b*b
            M[t] = BMat{v.limb, v.exp, v.sign, b, k * b * b, b * b, b * b};
        }
        int rc = fill_zero_batched(M[0], 1, k * b, b, p, st);
        if (rc == MP_OK) rc = fill_zero_batched(M[1], 1, k * b, b, p, st);
        const size_t plane = (size_t)k * b * b;
        for (int64_t i = 0; i < k && rc == MP_OK; ++i) {
            const mp_request_t &r = qs[i]->r;
            for (int src = 0; src < 2; ++src) {
                const int64_t rows = src ? r.l : r.m, cols = src ? r.n : r.l;
                const uint64_t *hl = src ? r.b_limb : r.a_limb;
                const int64_t *he = src ? r.b_exp : r.a_exp;
                const int8_t *hs = src ? r.b_sign : r.a_sign;
                if (!rows || !cols) continue;
                const BMat &D = M[src];
                for (int q = 0; q < L; ++q)
                    cudaMemcpy2DAsync(D.limb + q * plane + i * b * b, b * 8, hl + (size_t)q * rows * cols,
                                      cols * 8, cols * 8, rows, cudaMemcpyHostToDevice, st);
                cudaMemcpy2DAsync(D.exp + i * b * b, b * 8, he, cols * 8, cols * 8, rows,
                                  cudaMemcpyHostToDevice, st);
                cudaMemcpy2DAsync(D.sign + i * b * b, b, hs, cols, cols, rows, cudaMemcpyHostToDevice, st);
            }
        }
        if (rc == MP_OK && cudaGetLastError() != cudaSuccess) rc = MP_ERR_CUDA;
        if (rc == MP_OK) rc = gemm_block_batched(p, M[0], M[1], M[2], k, b, b, b, st);
        for (int64_t i = 0; i < k && rc == MP_OK; ++i) {
            const mp_request_t &r = qs[i]->r;
            if (!r.m || !r.n) continue;
            const BMat &D = M[2];
            for (int q = 0; q < L; ++q)
                cudaMemcpy2DAsync(r.c_limb + (size_t)q * r.m * r.n, r.n * 8, D.limb + q * plane + i * b * b,
                                  b * 8, r.n * 8, r.m, cudaMemcpyDeviceToHost, st);
            cudaMemcpy2DAsync(r.c_exp, r.n * 8, D.exp + i * b * b, b * 8, r.n * 8, r.m,
                              cudaMemcpyDeviceToHost, st);
            cudaMemcpy2DAsync(r.c_sign, r.n, D.sign + i * b * b, b, r.n, r.m, cudaMemcpyDeviceToHost, st);
        }
        if (rc == MP_OK && cudaGetLastError() != cudaSuccess) rc = MP_ERR_CUDA;
        cudaFreeAsync(mem, st);
        return rc;
    }

    // GEMMs of one precision as one group: every request's own operands,
    // result and workspace, its own recursion, and the leaves of all of
    // them in shared grouped launches (gemm_group)
    int run_group(const std::vector<Req *> &qs, cudaStream_t st)
    {
        const int p = qs[0]->r.prec;
        const size_t k = qs.size();
        std::vector<GroupGemm> items(k);
        std::vector<char *> mems(k, nullptr);
        int rc = MP_OK;
        for (size_t i = 0; i < k && rc == MP_OK; ++i) {
            const mp_request_t &r = qs[i]->r;
            const size_t sa = mat_size(p, r.m, r.l), sb = mat_size(p, r.l, r.n), sc = mat_size(p, r.m, r.n);
            const size_t sw = gemm_scratch_bytes(r.algo, r.m, r.l, r.n, r.cutoff, MP_PEEL, p);
            if (cudaMallocAsync((void **)&mems[i], sa + sb + sc + sw + 256, st) != cudaSuccess) {
                cudaGetLastError();
                mems[i] = nullptr;
                rc = MP_ERR_NOMEM;
                break;
            }
            mpmat_t A, B, C;
            mat_on(A, p, r.m, r.l, mems[i]);
            mat_on(B, p, r.l, r.n, mems[i] + sa);
            mat_on(C, p, r.m, r.n, mems[i] + sa + sb);
            rc = h2d(A, r.a_limb, r.a_exp, r.a_sign, st);
            if (rc == MP_OK) rc = h2d(B, r.b_limb, r.b_exp, r.b_sign, st);
            GroupGemm &g = items[i];
            g.algo = r.algo;
            g.cutoff = r.cutoff;
            g.m = r.m;
            g.l = r.l;
            g.n = r.n;
            g.A = BMat{A.limb, A.exp, A.sign, A.ld, A.plane, 0, 0};
            g.B = BMat{B.limb, B.exp, B.sign, B.ld, B.plane, 0, 0};
            g.C = BMat{C.limb, C.exp, C.sign, C.ld, C.plane, 0, 0};
            g.ws = (void *)(((uintptr_t)(mems[i] + sa + sb + sc) + 255) & ~(uintptr_t)255);
            g.ws_bytes = sw;
        }
        if (rc == MP_OK) rc = gemm_group(items.data(), (int)k, p, st);
        for (size_t i = 0; i < k && rc == MP_OK; ++i) {
            const mp_request_t &r = qs[i]->r;
            mpmat_t C;
            mat_on(C, p, r.m, r.n, mems[i] + mat_size(p, r.m, r.l) + mat_size(p, r.l, r.n));
            rc = d2h(C, r.c_limb, r.c_exp, r.c_sign, st);
        }
        for (char *m : mems)
            if (m) cudaFreeAsync(m, st);
        return rc;
    }

    // ------------------------------------------------------------- scheduler
    void retire_locked()
    {
        for (size_t u = 0; u < running.size();) {
            Unit *un = running[u];
            const cudaError_t q = cudaEventQuery(un->done);
            if (q == cudaErrorNotReady) { ++u; continue; }
            const auto now = Clock::now();
            const int st = (q == cudaSuccess && un->rc == MP_OK) ? MP_REQ_DONE : MP_REQ_FAILED;
            if (q != cudaSuccess) cudaGetLastError();
            for (Req *r : un->reqs) {
                const double ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
                finished.push_back({r->r.id, st, ms});
                delete r;
                ++n_completed;
                --outstanding;
            }
            used -= un->bytes;
            if (un->graph) un->graph->busy = false;
            busy[un->slot] = false;
            cudaEventDestroy(un->done);
            delete un;
            running[u] = running.back();
            running.pop_back();
        }
    }

    // choose the next unit to admit (queue lock held); nullptr if none fits
    Unit *pick_locked()
    {
        int slot = -1;
        for (size_t s = 0; s < busy.size(); ++s)
            if (!busy[s]) { slot = (int)s; break; }
        if (slot < 0) return nullptr;
        int scanned = 0;
        for (size_t i = 0; i < queue.size() && scanned < kLookAhead; ++i, ++scanned) {
            Req *h = queue[i];
            if (h->bucket > 0) {
                // gather same precision and bucket, in arrival order
                std::vector<size_t> idx;
                for (size_t j = i; j < queue.size() && (int)idx.size() < kMaxBatch; ++j) {
                    const Req *c = queue[j];
                    if (c->bucket == h->bucket && c->r.prec == h->r.prec) idx.push_back(j);
                }
                while (!idx.empty() &&
                       used + batch_bytes(h->r.prec, h->bucket, (int64_t)idx.size()) > budget)
                    idx.pop_back();
                if (idx.empty()) continue;
                Unit *u = new Unit;
                u->slot = slot;
                u->bytes = batch_bytes(h->r.prec, h->bucket, (int64_t)idx.size());
                for (size_t t = idx.size(); t-- > 0;) {
                    u->reqs.insert(u->reqs.begin(), queue[idx[t]]);
                    queue.erase(queue.begin() + (long)idx[t]);
                }
                return u;
            }
            // GEMMs of one precision and size class whose signatures have
            // not been seen (seen ones are candidates for the graph cache)
            // share their leaf launches; small Simple / Block requests that
            // wait beside them join as one leaf of their own shape
            const int64_t cls = group_class(h->r);
            if (cls > 0 && (graph_slots <= 0 || !seen.count(signature(h->r)))) {
                std::vector<size_t> idx;
                size_t need = 0;
                for (size_t j = i; j < queue.size() && j < i + kLookAhead && (int)idx.size() < kMaxGroup; ++j) {
                    const Req *c = queue[j];
                    if (c->r.prec != h->r.prec || group_class(c->r) != cls) continue;
                    if (graph_slots > 0 && seen.count(signature(c->r))) continue;
                    if (used + need + c->bytes > budget) continue;
                    idx.push_back(j);
                    need += c->bytes;
                }
                if (idx.size() >= 2) {
                    Unit *u = new Unit;
                    u->slot = slot;
                    u->group = true;
                    u->bytes = need;
                    for (size_t t = idx.size(); t-- > 0;) {
                        Req *q = queue[idx[t]];
                        if (graph_slots > 0) mark_seen(signature(q->r));
                        u->reqs.insert(u->reqs.begin(), q);
                        queue.erase(queue.begin() + (long)idx[t]);
                    }
                    return u;
                }
            }
            while (used + h->bytes > budget) {           // cached graphs give way to requests
                GraphEntry *v = lru_idle_locked();
                if (!v) break;
                evict_locked(v);
            }
            if (used + h->bytes <= budget) {
                Unit *u = new Unit;
                u->slot = slot;
                u->bytes = h->bytes;
                u->reqs.push_back(h);
                queue.erase(queue.begin() + (long)i);
                return u;
            }
        }
        return nullptr;
    }

    void loop()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            retire_locked();
            if (!finished.empty()) cv_done.notify_all();
            Unit *u = nullptr;
            while ((u = pick_locked()) != nullptr) {
                busy[u->slot] = true;
                used += u->bytes;
                peak = std::max(peak, used);
                for (Req *r : u->reqs) r->state = MP_REQ_RUNNING;
                running.push_back(u);
                const cudaStream_t st = streams[u->slot];
                lk.unlock();
                if (u->group)
                    u->rc = run_group(u->reqs, st);
                else if (u->reqs.size() > 1 || u->reqs[0]->bucket > 0)
                    u->rc = run_batch(u->reqs, u->reqs[0]->bucket, st);
                else
                    u->rc = run_request(u, st);
                cudaEventCreateWithFlags(&u->done, cudaEventDisableTiming);
                cudaEventRecord(u->done, st);
                lk.lock();
                if (u->reqs.size() > 1) {
                    ++n_batches;
                    n_batched_reqs += (int64_t)u->reqs.size();
                }
            }
            if (stop && queue.empty() && running.empty()) break;
            if (running.empty() && queue.empty())
                cv.wait(lk);
            else
                cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
};

extern "C" {

mp_server_t *mp_server_create(size_t budget_bytes, int slots)
{
    if (slots < 1 || slots > 64 || budget_bytes == 0) return nullptr;
    mp_server *s = new mp_server;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return nullptr; }
    s->budget = budget_bytes;
    s->streams.resize(slots);
    s->busy.assign(slots, false);
    for (int i = 0; i < slots; ++i)
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return nullptr;
        }
    s->th = std::thread([s] { s->loop(); });
    return s;
}

int mp_server_submit(mp_server_t *s, const mp_request_t *req)
{
    if (!s || !req) return MP_ERR_ARG;
    const mp_request_t &r = *req;
    if (r.prec < MP_PREC_MIN || r.prec > MP_PREC_MAX || r.m < 0 || r.l < 0 || r.n < 0) return MP_ERR_ARG;
    if (r.kind == MP_REQ_GEMM) {
        if (r.algo < MP_SIMPLE || r.algo > MP_WINOGRAD) return MP_ERR_ARG;
        if ((r.algo >= MP_STRASSEN) && r.cutoff < 0) return MP_ERR_ARG;
        if (r.m * r.l && (!r.a_limb || !r.a_exp || !r.a_sign)) return MP_ERR_ARG;
        if (r.l * r.n && (!r.b_limb || !r.b_exp || !r.b_sign)) return MP_ERR_ARG;
        if (r.m * r.n && (!r.c_limb || !r.c_exp || !r.c_sign)) return MP_ERR_ARG;
    } else if (r.kind == MP_REQ_LU_SOLVE) {
        if (r.algo < MP_SIMPLE || r.algo > MP_WINOGRAD || r.m < 1 || r.lu_panel < 0) return MP_ERR_ARG;
        if (!r.a_limb || !r.a_exp || !r.a_sign || !r.b_limb || !r.b_exp || !r.b_sign || !r.c_limb ||
            !r.c_exp || !r.c_sign)
            return MP_ERR_ARG;
    } else {
        return MP_ERR_ARG;
    }
    Req *q = new Req;
    q->r = r;
    q->t_submit = Clock::now();
    int64_t b = 0;
    if (batchable(r, &b)) {
        q->bucket = b;
        q->bytes = mp_server::batch_bytes(r.prec, b, 1);
    } else {
        q->bytes = s->footprint(r);
    }
    if (q->bytes > s->budget) {
        delete q;
        return MP_ERR_NOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.push_back(q);
        ++s->n_submitted;
        ++s->outstanding;
    }
    s->cv.notify_all();
    return MP_OK;
}

int mp_server_cancel(mp_server_t *s, int64_t id)
{
    if (!s) return MP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < s->queue.size(); ++i) {
        if (s->queue[i]->r.id == id) {
            Req *q = s->queue[i];
            s->queue.erase(s->queue.begin() + (long)i);
            const double ms =
                std::chrono::duration<double, std::milli>(Clock::now() - q->t_submit).count();
            s->finished.push_back({id, MP_REQ_CANCELLED, ms});
            --s->outstanding;
            delete q;
            s->cv_done.notify_all();
            return MP_OK;
        }
    }
    return MP_ERR_ARG;
}

int mp_server_poll(mp_server_t *s, int64_t *ids, int32_t *status, double *latency_ms, int max)
{
    if (!s || max < 0) return MP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    const int n = (int)std::min<size_t>((size_t)max, s->finished.size());
    for (int i = 0; i < n; ++i) {
        if (ids) ids[i] = s->finished[i].id;
        if (status) status[i] = s->finished[i].status;
        if (latency_ms) latency_ms[i] = s->finished[i].ms;
    }
    s->finished.erase(s->finished.begin(), s->finished.begin() + n);
    return n;
}

int mp_server_drain(mp_server_t *s)
{
    if (!s) return MP_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [s] { return s->outstanding == 0; });
    return MP_OK;
}

int mp_server_stats(mp_server_t *s, int64_t out[8])
{
    if (!s || !out) return MP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out[0] = s->n_submitted;
    out[1] = s->n_completed;
    out[2] = s->n_batches;
    out[3] = s->n_batched_reqs;
    out[4] = (int64_t)s->peak;
    out[5] = (int64_t)s->budget;
    out[6] = (int64_t)s->running.size();
    out[7] = (int64_t)s->queue.size();
    return MP_OK;
}

int mp_server_set_graphs(mp_server_t *s, int max_graphs)
{
    if (!s || max_graphs < 0 || max_graphs > 1024) return MP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->graph_slots = max_graphs;
    return MP_OK;
}

int mp_server_graph_stats(mp_server_t *s, int64_t out[4])
{
    if (!s || !out) return MP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out[0] = s->n_captures;
    out[1] = s->n_replays;
    out[2] = (int64_t)s->graphs.size();
    out[3] = (int64_t)s->graph_bytes;
    return MP_OK;
}

void mp_server_destroy(mp_server_t *s)
{
    if (!s) return;
    mp_server_drain(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    while (!s->graphs.empty()) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->evict_locked(s->graphs.back());
    }
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"

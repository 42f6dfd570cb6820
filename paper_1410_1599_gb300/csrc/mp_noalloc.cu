// mp_noalloc.cu -- mpgemm_noalloc: the Strassen / Winograd product with its
// recursion workspace in a fixed, statically allocated device array.
//
// Some callers cannot allocate device memory at the time they multiply:
// real-time or serving loops that must not touch an allocator (a cudaMalloc
// can synchronise the device and stall the loop), code running inside an
// allocator or memory-pool callback of a host framework (calling back into
// the allocator there can deadlock), and hosts whose device memory is all
// handed out up front by another owner (a new allocation fails).  This
// entry point takes nothing from any allocator: the temporaries of the
// recursion live in g_scratch below, which every GPU that loads the library
// holds (MP_NOALLOC_SCRATCH_BYTES) until the process exits, and range
// errors go to the static status word g_status, which mp_sync_status()
// reads.
#include <cstdio>
#include <mutex>

#include "../../include/mpgemm.h"
#include "mp_internal.h"

namespace mpg {
int gemm_in_block(int algo, int cutoff, int policy, int64_t m, int64_t l, int64_t n, int p,
                  const mpmat_t *A, const mpmat_t *B, mpmat_t *C, void *base, size_t bytes,
                  DevStatus *st, cudaStream_t s);
size_t gemm_scratch_bytes(int algo, int64_t m, int64_t l, int64_t n, int cutoff, int policy, int p);
int resolve_cutoff(int cutoff, int p);
bool gemm_args_ok(int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo, int32_t cutoff,
                  const mpmat_t *A, const mpmat_t *B, const mpmat_t *C);
cudaStream_t current_stream();
int current_odd_policy();
}  // namespace mpg

namespace {

// The shared scratch and status word.  In host code these names denote
// host-side stand-ins, not device memory: kernels must be given the device
// addresses obtained with cudaGetSymbolAddress (see device_ptrs).
static __device__ __align__(256) unsigned char g_scratch[MP_NOALLOC_SCRATCH_BYTES];
static __device__ mpg::DevStatus g_status = {0u, 0u, INT64_MAX, 0ull};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_base[kMaxDevices] = {};
mpg::DevStatus *g_st[kMaxDevices] = {};

// Device addresses of g_scratch and g_status on the current device, looked
// up once per device (the first call on a device does this set-up).
int device_ptrs(void **base, mpg::DevStatus **st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr, *q = nullptr;
        cudaError_t rc = cudaGetSymbolAddress(&p, g_scratch);
        if (rc == cudaSuccess) rc = cudaGetSymbolAddress(&q, g_status);
        if (rc != cudaSuccess || !p || !q) {
            cudaGetLastError();
            return MP_ERR_CUDA;
        }
        g_st[dev] = static_cast<mpg::DevStatus *>(q);
        g_base[dev] = p;
    }
    *base = g_base[dev];
    *st = g_st[dev];
    return MP_OK;
}

}  // namespace

namespace mpg {
unsigned noalloc_take_flags()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0u;
    DevStatus *st;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        st = g_st[dev];
    }
    if (!st) return 0u;
    DevStatus h{};
    if (cudaMemcpy(&h, st, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return 0u;
    if (h.flags) {
        const DevStatus init{0u, 0u, INT64_MAX, 0ull};
        cudaMemcpy(st, &init, sizeof init, cudaMemcpyHostToDevice);
    }
    return h.flags;
}
}  // namespace mpg

extern "C" int mpgemm_noalloc(int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo,
                              int32_t cutoff, const mpmat_t *A, const mpmat_t *B, mpmat_t *C)
{
    using namespace mpg;
    // the exact-dot and split forms keep their own large buffers: not offered here
    if (algo == MP_EXACT || algo == MP_SPLIT) return MP_ERR_UNSUPPORTED;
    if (!gemm_args_ok(m, l, n, prec, algo, cutoff, A, B, C)) return MP_ERR_ARG;
    cutoff = resolve_cutoff(cutoff, prec);
    const int policy = current_odd_policy();
    const size_t need = gemm_scratch_bytes(algo, m, l, n, cutoff, policy, prec);
    if (need > (size_t)MP_NOALLOC_SCRATCH_BYTES) return MP_ERR_SCRATCH;
    if (m == 0 || n == 0) return MP_OK;
    void *base = nullptr;
    DevStatus *st = nullptr;
    const int rc = device_ptrs(&base, &st);
    if (rc != MP_OK) return rc;
    return gemm_in_block(algo, cutoff, policy, m, l, n, prec, A, B, C, base,
                         (size_t)MP_NOALLOC_SCRATCH_BYTES, st, current_stream());
}

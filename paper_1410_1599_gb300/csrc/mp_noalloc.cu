// mp_noalloc.cu -- mpgemm_noalloc: the Strassen / Winograd product with its
// recursion workspace in a fixed, statically allocated device array.
//
// Some callers cannot allocate device memory at the time they multiply: code
// running while a CUDA stream is being captured into a graph (an allocation
// there would break or stall the capture), real-time or serving loops that
// must not touch the allocator, and hosts whose device memory is handed out
// up front by another owner.  This entry point takes nothing from any
// allocator: the temporaries of the recursion live in g_scratch below, which
// every GPU that loads the library holds (MP_NOALLOC_SCRATCH_BYTES) until the
// process exits.
#include <cstdio>
#include <mutex>

#include "../../include/mpgemm.h"
#include "mp_internal.h"

namespace mpg {
int gemm_in_block(int algo, int cutoff, int policy, int64_t m, int64_t l, int64_t n, int p,
                  const mpmat_t *A, const mpmat_t *B, mpmat_t *C, void *base, size_t bytes,
                  cudaStream_t s);
size_t gemm_scratch_bytes(int algo, int64_t m, int64_t l, int64_t n, int cutoff, int policy, int p);
int resolve_cutoff(int cutoff, int p);
bool gemm_args_ok(int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo, int32_t cutoff,
                  const mpmat_t *A, const mpmat_t *B, const mpmat_t *C);
cudaStream_t current_stream();
int current_odd_policy();
}  // namespace mpg

namespace {

// The shared scratch.  In host code `g_scratch` names a host-side stand-in,
// not device memory: kernels must be given the device address obtained with
// cudaGetSymbolAddress (see scratch_base).
static __device__ __align__(256) unsigned char g_scratch[MP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_base[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device (the first call on a device does this set-up).
int scratch_base(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        const cudaError_t rc = cudaGetSymbolAddress(&p, g_scratch);
        if (rc != cudaSuccess || !p) {
            cudaGetLastError();
            return MP_ERR_CUDA;
        }
        g_base[dev] = p;
    }
    *out = g_base[dev];
    return MP_OK;
}

}  // namespace

extern "C" int mpgemm_noalloc(int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo,
                              int32_t cutoff, const mpmat_t *A, const mpmat_t *B, mpmat_t *C)
{
    using namespace mpg;
    if (!gemm_args_ok(m, l, n, prec, algo, cutoff, A, B, C)) return MP_ERR_ARG;
    cutoff = resolve_cutoff(cutoff, prec);
    const int policy = current_odd_policy();
    const size_t need = gemm_scratch_bytes(algo, m, l, n, cutoff, policy, prec);
    if (need > (size_t)MP_NOALLOC_SCRATCH_BYTES) return MP_ERR_SCRATCH;
    if (m == 0 || n == 0) return MP_OK;
    void *base = nullptr;
    const int rc = scratch_base(&base);
    if (rc != MP_OK) return rc;
    return gemm_in_block(algo, cutoff, policy, m, l, n, prec, A, B, C, base,
                         (size_t)MP_NOALLOC_SCRATCH_BYTES, current_stream());
}

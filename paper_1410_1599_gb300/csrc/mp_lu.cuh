// mp_lu.cuh -- kernels of the blocked right-looking LU with partial pivoting
// and the triangular solves (arXiv 1410.1599 Sec. 4), one instantiation per
// word-capacity class W (lu_w*.cu).
#pragma once
#include "mp_kernels.cuh"

namespace mpg {

// |x| > |y| on loaded numbers (zero is the smallest magnitude)
template <int W>
MP_DEV bool absgreater(const Mp<W> &x, const Mp<W> &y)
{
    return cmpabs<W>(x, y) > 0;
}

// One CTA: pivot = first row i in [k, n) of largest |a_ik|; record it, then
// exchange rows k and pivot over all n columns.  A zero pivot column is
// recorded (smallest such column wins) and nothing is exchanged.
template <int W>
__global__ void __launch_bounds__(1024) lu_pivot_kernel(BMat A, int64_t n, int64_t k, int64_t *piv,
                                                        int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    __shared__ int64_t s_row[1024];
    __shared__ int64_t s_best;
    const int tid = threadIdx.x, nt = blockDim.x;
    // per thread: best candidate by (exponent, then limbs, then lowest row)
    int64_t best = -1;
    Mp<W> bx, x;
    set_zero<W>(bx, 0u);
    for (int64_t i = k + tid; i < n; i += nt) {
        ld_rw<W>(x, A, 0, i, k, rs.L);
        if (best < 0 || absgreater<W>(x, bx)) {
            best = i;
            bx = x;
        }
    }
    s_row[tid] = best;
    __syncthreads();
    // tree reduction: compare through global memory reloads (rows are few)
    for (int stride = nt / 2; stride > 0; stride >>= 1) {
        if (tid < stride) {
            const int64_t ra = s_row[tid], rb = s_row[tid + stride];
            if (rb >= 0) {
                bool take = false;
                if (ra < 0) take = true;
                else {
                    Mp<W> xa, xb;
                    ld_rw<W>(xa, A, 0, ra, k, rs.L);
                    ld_rw<W>(xb, A, 0, rb, k, rs.L);
                    const int c = cmpabs<W>(xb, xa);
                    take = c > 0 || (c == 0 && rb < ra);
                }
                if (take) s_row[tid] = rb;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int64_t pr = s_row[0] < 0 ? k : s_row[0];
        Mp<W> v;
        ld_rw<W>(v, A, 0, pr, k, rs.L);
        piv[k] = pr;
        if (v.e == EXP_ZERO) {
            atomicOr(&status->flags, ST_SINGULAR);
            atomicMin(&status->singular_col, (long long)k);
            s_best = k;   // no exchange
        } else {
            s_best = pr;
        }
    }
    __syncthreads();
    const int64_t pr = s_best;
    if (pr == k) return;
    const int L = rs.L;
    for (int64_t c = tid; c < n; c += nt) {
        for (int q = 0; q < L; ++q) {
            uint64_t *a = A.limb + (int64_t)q * A.plane + k * A.ld + c;
            uint64_t *b = A.limb + (int64_t)q * A.plane + pr * A.ld + c;
            const uint64_t t = *a;
            *a = *b;
            *b = t;
        }
        int64_t *ea = A.exp + k * A.ld + c, *eb = A.exp + pr * A.ld + c;
        const int64_t te = *ea;
        *ea = *eb;
        *eb = te;
        int8_t *sa = A.sign + k * A.ld + c, *sb = A.sign + pr * A.ld + c;
        const int8_t ts = *sa;
        *sa = *sb;
        *sb = ts;
    }
}

// l_ik = RN(a_ik / a_kk) for i in (k, n); a zero a_kk (already reported by
// the pivot step) leaves the column untouched
template <int W>
__global__ void lu_divide_kernel(BMat A, int64_t n, int64_t k, int p)
{
    const RoundSpec rs = make_spec<W>(p);
    Mp<W> d, x, q;
    ld_rw<W>(d, A, 0, k, k, rs.L);
    if (d.e == EXP_ZERO) return;
    for (int64_t i = k + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        ld_rw<W>(x, A, 0, i, k, rs.L);
        div<W>(q, x, d, rs);
        st<W>(q, A, 0, i, k, rs.L);
    }
}

// a_ij = RN(a_ij - RN(a_ik a_kj)) for i in [r0, r1), j in [c0, c1): one
// elimination step of the panel (column k) or of the U12 solve (row s = k)
template <int W>
__global__ void lu_rank1_kernel(BMat A, int64_t k, int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                                int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int64_t w = c1 - c0, total = (r1 - r0) * w;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = r0 + t / w, j = c0 + t % w;
        Mp<W> l, u, y, z;
        ld_rw<W>(l, A, 0, i, k, rs.L);
        ld_rw<W>(u, A, 0, k, j, rs.L);
        ld_rw<W>(y, A, 0, i, j, rs.L);
        mul<W>(z, l, u, rs);
        add<W>(y, y, z, 1u, rs);
        bad |= st<W>(y, A, 0, i, j, rs.L);
    }
    if (bad) flag(status, ST_RANGE);
}

// One CTA: x = U^-1 L^-1 P b, both substitutions column by column.  y is an
// n x 1 work vector; x receives the solution.
template <int W>
__global__ void __launch_bounds__(1024) lu_solve_kernel(BMat LU, int64_t n, const int64_t *piv,
                                                        BMat b, BMat y, BMat x, int64_t *perm,
                                                        int p, DevStatus *status)
{
    const RoundSpec rs = make_spec<W>(p);
    const int tid = threadIdx.x, nt = blockDim.x;
    // permutation of the row exchanges, applied in order
    for (int64_t i = tid; i < n; i += nt) perm[i] = i;
    __syncthreads();
    if (tid == 0) {
        for (int64_t k = 0; k < n; ++k) {
            const int64_t q = piv[k];
            const int64_t t = perm[k];
            perm[k] = perm[q];
            perm[q] = t;
        }
    }
    __syncthreads();
    Mp<W> v, l, u, z;
    for (int64_t i = tid; i < n; i += nt) {
        ld_rw<W>(v, b, 0, perm[i], 0, rs.L);
        st<W>(v, y, 0, i, 0, rs.L);
    }
    __syncthreads();
    // forward: unit lower
    for (int64_t j = 0; j < n; ++j) {
        Mp<W> yj;
        ld_rw<W>(yj, y, 0, j, 0, rs.L);
        for (int64_t i = j + 1 + tid; i < n; i += nt) {
            ld_rw<W>(l, LU, 0, i, j, rs.L);
            ld_rw<W>(v, y, 0, i, 0, rs.L);
            mul<W>(z, l, yj, rs);
            add<W>(v, v, z, 1u, rs);
            st<W>(v, y, 0, i, 0, rs.L);
        }
        __syncthreads();
    }
    // backward: x_j = y_j / u_jj, then eliminate x_j from rows i < j
    __shared__ int s_zero;
    if (tid == 0) s_zero = 0;
    __syncthreads();
    for (int64_t j = n - 1; j >= 0; --j) {
        if (tid == 0) {
            ld_rw<W>(v, y, 0, j, 0, rs.L);
            ld_rw<W>(u, LU, 0, j, j, rs.L);
            if (u.e == EXP_ZERO) {
                s_zero = 1;
                set_zero<W>(z, 0u);
            } else {
                div<W>(z, v, u, rs);
            }
            st<W>(z, x, 0, j, 0, rs.L);
        }
        __syncthreads();
        Mp<W> xj;
        ld_rw<W>(xj, x, 0, j, 0, rs.L);
        for (int64_t i = tid; i < j; i += nt) {
            ld_rw<W>(u, LU, 0, i, j, rs.L);
            ld_rw<W>(v, y, 0, i, 0, rs.L);
            mul<W>(z, u, xj, rs);
            add<W>(v, v, z, 1u, rs);
            st<W>(v, y, 0, i, 0, rs.L);
        }
        __syncthreads();
    }
    if (tid == 0 && s_zero) atomicOr(&status->flags, ST_SINGULAR);
}

// ================================================================ launchers
template <int W>
void launch_lu_pivot(BMat A, int64_t n, int64_t k, int64_t *piv, int p, DevStatus *st,
                     cudaStream_t s)
{
    lu_pivot_kernel<W><<<1, (W <= 16) ? 1024 : 256, 0, s>>>(A, n, k, piv, p, st);
}

template <int W>
void launch_lu_divide(BMat A, int64_t n, int64_t k, int p, cudaStream_t s)
{
    const int64_t rows = n - k - 1;
    if (rows <= 0) return;
    lu_divide_kernel<W><<<grid_for(rows, 64), 64, 0, s>>>(A, n, k, p);
}

template <int W>
void launch_lu_rank1(BMat A, int64_t k, int64_t r0, int64_t r1, int64_t c0, int64_t c1, int p,
                     DevStatus *st, cudaStream_t s)
{
    const int64_t total = (r1 - r0) * (c1 - c0);
    if (r1 <= r0 || c1 <= c0) return;
    lu_rank1_kernel<W><<<grid_for(total, 128), 128, 0, s>>>(A, k, r0, r1, c0, c1, p, st);
}

template <int W>
void launch_lu_solve(BMat LU, int64_t n, const int64_t *piv, BMat b, BMat y, BMat x,
                     int64_t *perm, int p, DevStatus *st, cudaStream_t s)
{
    const int threads = (W <= 16) ? 1024 : (W == 32 ? 512 : 256);
    lu_solve_kernel<W><<<1, threads, 0, s>>>(LU, n, piv, b, y, x, perm, p, st);
}

#define MPG_INSTANTIATE_LU(W)                                                                   \
    template void launch_lu_pivot<W>(BMat, int64_t, int64_t, int64_t *, int, DevStatus *,       \
                                     cudaStream_t);                                             \
    template void launch_lu_divide<W>(BMat, int64_t, int64_t, int, cudaStream_t);               \
    template void launch_lu_rank1<W>(BMat, int64_t, int64_t, int64_t, int64_t, int64_t, int,    \
                                     DevStatus *, cudaStream_t);                                \
    template void launch_lu_solve<W>(BMat, int64_t, const int64_t *, BMat, BMat, BMat,          \
                                     int64_t *, int, DevStatus *, cudaStream_t);

}  // namespace mpg

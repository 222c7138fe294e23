// One-time set-up of the pump matrix (Eq. 2), its noise factor L L^T = W for the
// correlated noise chi = L eta (Sec. S1), and the spectrum diagnostics w_max,
// w_min (Eq. 3 and the w_min estimate below it). All FP64 on the device.
#include <math.h>

#include "twa_internal.cuh"

namespace twa {
namespace {

// W_ij = w / (|i-j| + 1)^alpha (Eq. 2); alpha = +inf -> w delta_ij.
__global__ void k_pump_matrix(double* W, int64_t N, double alpha, double w) {
    const int64_t n2 = N * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N, j = e - i * N;
        const int64_t d = i > j ? i - j : j - i;
        double v;
        if (isinf(alpha)) v = (d == 0) ? w : 0.0;
        else if (alpha == 0.0) v = w;
        else v = w / pow((double)(d + 1), alpha);
        W[e] = v;
    }
}

// Noise factors with a closed form: rank one for alpha = 0 (L[:,0] = sqrt w),
// sqrt(w) I for alpha = +inf, zero for w = 0.
__global__ void k_special_factor(double* L, int64_t N, int mode, double sw) {
    const int64_t n2 = N * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N, j = e - i * N;
        double v = 0.0;
        if (mode == 0 && j == 0) v = sw;
        if (mode == 1 && i == j) v = sw;
        L[e] = v;
    }
}

constexpr int NB = 32;  // Cholesky panel width

// Unblocked Cholesky of the (already updated) diagonal block A[k:k+kb, k:k+kb],
// one thread per entry. A pivot <= 0 is counted; with `clip` the column is
// zeroed, otherwise it is zeroed too (so the factor stays finite) and the host
// reports TWA_ENOTPSD.
__global__ void k_potrf_diag(double* A, int64_t lda, int64_t k, int kb, double* piv,
                             unsigned long long* flags) {
    __shared__ double a[NB][NB + 1];
    const int r = threadIdx.y, c = threadIdx.x;
    if (r < kb && c < kb) a[r][c] = A[(k + r) * lda + k + c];
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        const double p = a[j][j];
        const bool ok = p > 0.0;
        __syncthreads();
        if (r == 0 && c == 0) {
            piv[k + j] = p;
            if (!ok) {
                if (atomicAdd(&flags[FLAG_NOTPSD], 1ull) == 0ull) flags[FLAG_NOTPSD_IDX] = (unsigned long long)(k + j + 1);
            }
        }
        const double l = ok ? sqrt(p) : 0.0;
        if (c == j && r >= j && r < kb) a[r][j] = (r == j) ? l : (ok ? a[r][j] / l : 0.0);
        __syncthreads();
        if (r > j && c > j && c <= r && r < kb) a[r][c] -= a[r][j] * a[c][j];
        __syncthreads();
    }
    if (r < kb && c < kb) A[(k + r) * lda + k + c] = (c <= r) ? a[r][c] : 0.0;
}

// Panel solve: rows r >= k+kb of A[:, k:k+kb] <- A[:, k:k+kb] L_kk^{-T}.
__global__ void k_trsm_panel(double* A, int64_t lda, int64_t k, int kb, int64_t N) {
    __shared__ double l[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        l[r][c] = (r < kb && c < kb) ? A[(k + r) * lda + k + c] : 0.0;
    }
    __syncthreads();
    const int64_t row = k + kb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= N) return;
    double x[NB];
    double* a = A + row * lda + k;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j < kb) {
            double s = a[j];
            for (int p = 0; p < j; ++p) s -= x[p] * l[j][p];
            x[j] = (l[j][j] > 0.0) ? s / l[j][j] : 0.0;
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < kb) a[j] = x[j];
}

__global__ void k_zero_upper(double* L, int64_t N) {
    const int64_t n2 = N * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N, j = e - i * N;
        if (j > i) L[e] = 0.0;
    }
}

__global__ void k_min_reduce(const double* v, int64_t n, double* out) {
    __shared__ double sm[256];
    double m = INFINITY;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) m = fmin(m, v[e]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] = fmin(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

// Squared Frobenius norms of W - R and of W (R = L L^T), one block:
// out[0] = sum (W - R)^2, out[1] = sum W^2.
__global__ void k_residual_norms(const double* W, const double* R, int64_t n2, double* out) {
    __shared__ double sd[256], sw[256];
    double d = 0.0, ww = 0.0;
    for (int64_t e = threadIdx.x; e < n2; e += blockDim.x) {
        const double x = W[e] - R[e];
        d += x * x;
        ww += W[e] * W[e];
    }
    sd[threadIdx.x] = d;
    sw[threadIdx.x] = ww;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sd[threadIdx.x] += sd[threadIdx.x + s];
            sw[threadIdx.x] += sw[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sd[0];
        out[1] = sw[0];
    }
}

// ---------------------------------------------------------------------------
// Lanczos for the extreme eigenvalues of W. y = W v, one warp per row.
__global__ void k_matvec(const double* W, const double* v, double* y, int64_t N) {
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= N) return;
    double s = 0.0;
    for (int64_t j = lane; j < N; j += 32) s += W[row * N + j] * v[j];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
}

// One block: out = a . b
__global__ void k_dot(const double* a, const double* b, int64_t n, double* out) {
    __shared__ double sm[1024];
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s += a[e] * b[e];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

// Lanczos update with y = W v_j already computed:
// alpha_j = y.v_j; y -= alpha_j v_j + beta_{j-1} v_{j-1}; beta_j = |y|; v_{j+1} = y / beta_j.
// Single block so the two reductions stay in one launch.
__global__ void k_lanczos_update(double* y, const double* v, const double* vprev, double* vnext,
                                 double* alph, double* bet, int j, int64_t N) {
    __shared__ double sm[1024];
    __shared__ double s_a, s_b;
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < N; e += blockDim.x) s += y[e] * v[e];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) s_a = sm[0];
    __syncthreads();
    const double a = s_a, bp = (j > 0) ? bet[j - 1] : 0.0;
    s = 0.0;
    for (int64_t e = threadIdx.x; e < N; e += blockDim.x) {
        const double r = y[e] - a * v[e] - (j > 0 ? bp * vprev[e] : 0.0);
        y[e] = r;
        s += r * r;
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) s_b = sqrt(sm[0]);
    __syncthreads();
    const double b = s_b;
    for (int64_t e = threadIdx.x; e < N; e += blockDim.x) vnext[e] = (b > 0.0) ? y[e] / b : 0.0;
    if (threadIdx.x == 0) {
        alph[j] = a;
        bet[j] = b;
    }
}

// Number of eigenvalues of the leading k x k Lanczos tridiagonal below x (Sturm
// sequence of the LDL^T pivots). The recurrence is cut at the first beta below
// tol (an invariant subspace) by the caller.
__device__ int sturm_count(const double* a, const double* b, int k, double x) {
    int cnt = 0;
    double d = 1.0;
    for (int j = 0; j < k; ++j) {
        const double bb = (j > 0) ? b[j - 1] * b[j - 1] : 0.0;
        d = a[j] - x - (j > 0 ? bb / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// Extreme eigenvalues of the tridiagonal by multisection of Sturm counts: in
// each round the block's threads evaluate the count at as many interior points
// of the bracket, which then shrinks to the sub-interval where the count first
// reaches the target (1 for the smallest eigenvalue, k for the largest): a
// factor blockDim + 1 per round, so 8 rounds reach FP64 resolution.
__global__ void __launch_bounds__(1024) k_tridiag_extremes(const double* a, const double* b, int kmax,
                                                           double* out) {
    __shared__ int s_k, s_first;
    __shared__ double s_lo, s_hi;
    if (threadIdx.x == 0) {
        double amax = 0.0;
        for (int j = 0; j < kmax; ++j) amax = fmax(amax, fabs(a[j]));
        int k = kmax;
        for (int j = 0; j < kmax - 1; ++j)
            if (b[j] <= 1e-12 * fmax(amax, 1e-300)) { k = j + 1; break; }
        double lo = INFINITY, hi = -INFINITY;   // Gershgorin bracket
        for (int j = 0; j < k; ++j) {
            const double r = (j > 0 ? fabs(b[j - 1]) : 0.0) + (j < k - 1 ? fabs(b[j]) : 0.0);
            lo = fmin(lo, a[j] - r);
            hi = fmax(hi, a[j] + r);
        }
        s_k = k;
        s_lo = lo;
        s_hi = hi;
    }
    __syncthreads();
    const int k = s_k;
    const double T1 = (double)(blockDim.x + 1);
    for (int which = 0; which < 2; ++which) {
        const int target = (which == 0) ? 1 : k;
        double l = s_lo, h = s_hi;
        for (int round = 0; round < 8; ++round) {
            const double x = l + (h - l) * (double)(threadIdx.x + 1) / T1;
            if (threadIdx.x == 0) s_first = blockDim.x;
            __syncthreads();
            if (sturm_count(a, b, k, x) >= target) atomicMin(&s_first, (int)threadIdx.x);
            __syncthreads();
            const int f = s_first;
            // the count reaches the target in (x_{f-1}, x_f], x_{-1} = l, x_T = h
            const double nl = (f == 0) ? l : l + (h - l) * (double)f / T1;
            const double nh = (f == (int)blockDim.x) ? h : l + (h - l) * (double)(f + 1) / T1;
            l = nl;
            h = nh;
            __syncthreads();
        }
        if (threadIdx.x == 0) out[which == 0 ? 1 : 0] = 0.5 * (l + h);
    }
}

__global__ void k_rescale(double* v, int64_t N, const double* nrm2) {
    const double s = 1.0 / sqrt(*nrm2);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
        v[e] *= s;
}

__global__ void k_lanczos_start(double* v, int64_t N) {
    // a fixed, dense start vector with no symmetry of the chain
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = (1.0 + 0.37 * sin(1.3 * (double)e + 0.2)) / sqrt((double)N);
}

}  // namespace

int setup_pump(twa_ctx* c) {
    const int64_t N = c->N;
    cudaStream_t st = c->stream;
    const int grid = (int)((N * N + 255) / 256 > 4096 ? 4096 : (N * N + 255) / 256);
    k_pump_matrix<<<grid, 256, 0, st>>>(c->W64, N, c->alpha, c->w);
    TWA_CUDA(c, cudaGetLastError());

    Scratch<double> piv_buf(c, st);
    TWA_CUDA(c, piv_buf.alloc(sizeof(double) * (N + 8)));
    double* piv = piv_buf.p;
    c->clipped = 0;
    c->factor_residual = 0.0;
    if (c->w == 0.0 || c->alpha == 0.0 || isinf(c->alpha)) {
        const int mode = (c->w == 0.0) ? 2 : (c->alpha == 0.0 ? 0 : 1);
        k_special_factor<<<grid, 256, 0, st>>>(c->L64, N, mode, sqrt(c->w));
        TWA_CUDA(c, cudaGetLastError());
        c->min_pivot = (mode == 1) ? c->w : (mode == 0 ? (N == 1 ? c->w : 0.0) : 0.0);
    } else {
        TWA_CUDA(c, cudaMemcpyAsync(c->L64, c->W64, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, st));
        for (int64_t k = 0; k < N; k += NB) {
            const int kb = (int)((N - k) < NB ? (N - k) : NB);
            k_potrf_diag<<<1, dim3(NB, NB), 0, st>>>(c->L64, N, k, kb, piv, c->d_flags);
            const int64_t rest = N - k - kb;
            if (rest > 0) {
                k_trsm_panel<<<(unsigned)((rest + 127) / 128), 128, 0, st>>>(c->L64, N, k, kb, N);
                double* P = c->L64 + (k + kb) * N + k;
                gemm_f64(P, N, P, N, c->L64 + (k + kb) * N + (k + kb), N, rest, rest, kb, -1.0, 1.0,
                         false, true, st);
            }
        }
        TWA_CUDA(c, cudaGetLastError());
        k_zero_upper<<<grid, 256, 0, st>>>(c->L64, N);
        k_min_reduce<<<1, 256, 0, st>>>(piv, N, piv + N);
        TWA_CUDA(c, cudaGetLastError());
        unsigned long long fl[FLAG_COUNT];
        TWA_CUDA(c, cudaMemcpyAsync(&c->min_pivot, piv + N, sizeof(double), cudaMemcpyDeviceToHost, st));
        TWA_CUDA(c, cudaMemcpyAsync(fl, c->d_flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
        TWA_CUDA(c, cudaStreamSynchronize(st));
        if (fl[FLAG_NOTPSD] > 0) {
            c->clipped = (int64_t)fl[FLAG_NOTPSD];
            if (!c->opts.clip_negative) {
                return set_error(c, TWA_ENOTPSD,
                                 "pump matrix not positive definite: pivot " +
                                     std::to_string((long long)fl[FLAG_NOTPSD_IDX] - 1) + " <= 0 (" +
                                     std::to_string((long long)fl[FLAG_NOTPSD]) + " such pivots)");
            }
            TWA_CUDA(c, cudaMemsetAsync(c->d_flags + FLAG_NOTPSD, 0, 2 * sizeof(unsigned long long), st));
            // clipping zeroes the column of each non-positive pivot (it is not an
            // eigenvalue clip): report how far L L^T is from W, ||W - L L^T||_F / ||W||_F
            Scratch<double> r_buf(c, st);
            TWA_CUDA(c, r_buf.alloc(sizeof(double) * (N * N + 2)));
            double* R = r_buf.p;
            TWA_CUDA(c, cudaMemsetAsync(R, 0, sizeof(double) * N * N, st));
            gemm_f64(c->L64, N, c->L64, N, R, N, N, N, N, 1.0, 0.0, true, false, st);
            k_residual_norms<<<1, 256, 0, st>>>(c->W64, R, N * N, R + N * N);
            double nr[2] = {0.0, 0.0};
            const cudaError_t e1 = cudaGetLastError();
            const cudaError_t e2 = cudaMemcpyAsync(nr, R + N * N, sizeof(nr), cudaMemcpyDeviceToHost, st);
            const cudaError_t e3 = cudaStreamSynchronize(st);
            TWA_CUDA(c, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3));
            c->factor_residual = nr[1] > 0.0 ? sqrt(nr[0] / nr[1]) : 0.0;
        }
    }

    // spectrum: Lanczos on W
    // the low end of the spectrum is dense for long-range pumps, so the Krylov
    // space is taken large (the full space for N <= 1024)
    const int kmax = (int)(N < 1024 ? N : 1024);
    Scratch<double> lz_buf(c, st);
    TWA_CUDA(c, lz_buf.alloc(sizeof(double) * (4 * N + 2 * kmax + 8)));
    double* lz = lz_buf.p;
    double *v0 = lz, *v1 = lz + N, *v2 = lz + 2 * N, *y = lz + 3 * N;
    double *al = lz + 4 * N, *be = al + kmax, *ext = be + kmax;
    k_lanczos_start<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(v1, N);
    k_dot<<<1, 1024, 0, st>>>(v1, v1, N, ext + 2);
    k_rescale<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(v1, N, ext + 2);
    TWA_CUDA(c, cudaMemsetAsync(v0, 0, sizeof(double) * N, st));
    double *vp = v0, *vc = v1, *vn = v2;
    for (int j = 0; j < kmax; ++j) {
        k_matvec<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(c->W64, vc, y, N);
        k_lanczos_update<<<1, 1024, 0, st>>>(y, vc, vp, vn, al, be, j, N);
        double* t = vp; vp = vc; vc = vn; vn = t;
    }
    k_tridiag_extremes<<<1, 1024, 0, st>>>(al, be, kmax, ext);
    TWA_CUDA(c, cudaGetLastError());
    double e2[2];
    TWA_CUDA(c, cudaMemcpyAsync(e2, ext, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    TWA_CUDA(c, cudaStreamSynchronize(st));
    c->w_max = e2[0];
    c->w_min = e2[1];
    TWA_CUDA(c, cudaStreamSynchronize(st));
    return TWA_OK;
}

}  // namespace twa

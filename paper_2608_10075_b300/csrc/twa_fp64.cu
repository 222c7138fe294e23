// Plain FP64 GPU path: every step of Eq. S1 in double precision, with a SIMT
// DFMA GEMM for the two contractions (pump field W.s, correlated noise L.eta)
// and elementwise Heun kernels. It is the precision reference for the
// tensor-core path and the comparison point for its speed.
//
// Layouts: xy [2M][N] with row 2m = s^x of trajectory m and row 2m+1 = s^y;
// z [M][N]. A contraction C[n][i] = sum_k A[i][k] B[n][k] then maps the state
// rows n straight onto output rows of the same layout.
#include <math.h>

#include "twa_internal.cuh"

namespace twa {
namespace {

constexpr int GT = 64;   // GEMM tile (rows i and rows n)
constexpr int GK = 16;   // K per smem stage

// C[n][i] = alpha * sum_k A[i][k] B[n][k] + beta * C[n][i]. `tri_a`: A is lower
// triangular, so k stops at the end of the i tile. `lower_only`: skip tiles
// strictly above the diagonal n >= i (symmetric rank-k update).
__global__ void __launch_bounds__(256) k_gemm_f64(const double* __restrict__ A, int64_t lda,
                                                  const double* __restrict__ B, int64_t ldb,
                                                  double* __restrict__ C, int64_t ldc, int64_t n_i, int64_t n_n,
                                                  int64_t K, double alpha, double beta, int tri_a,
                                                  int lower_only) {
    const int64_t i0 = (int64_t)blockIdx.x * GT, n0 = (int64_t)blockIdx.y * GT;
    if (lower_only && n0 + GT - 1 < i0) return;
    int64_t kend = K;
    if (tri_a && i0 + GT < kend) kend = i0 + GT;
    __shared__ double As[GK][GT + 2];
    __shared__ double Bs[GK][GT + 2];
    const int tid = threadIdx.x;
    const int ti = tid & 15, tn = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int64_t k0 = 0; k0 < kend; k0 += GK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int row = e >> 4, kk = e & 15;
            const int64_t k = k0 + kk;
            As[kk][row] = (i0 + row < n_i && k < kend) ? A[(i0 + row) * lda + k] : 0.0;
            Bs[kk][row] = (n0 + row < n_n && k < kend) ? B[(n0 + row) * ldb + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ti * 4 + q];
                b[q] = Bs[kk][tn * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(b[p], a[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t n = n0 + tn * 4 + p;
        if (n >= n_n) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + ti * 4 + q;
            if (i >= n_i) continue;
            if (lower_only && n < i) continue;
            double* cp = C + n * ldc + i;
            *cp = alpha * acc[p][q] + (beta != 0.0 ? beta * *cp : 0.0);
        }
    }
}

// Discrete-Wigner initial state (Sec. S1, item 3): x, y = +-1, z = init_sz.
__global__ void k_init_f64(double* xy, double* z, int64_t M, int64_t N, uint64_t seed, double init_sz,
                           int64_t m0) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N;
    double sx, sy;
    init_signs(seed, (uint32_t)(m0 + m), (uint32_t)i, sx, sy);
    xy[(2 * m) * N + i] = sx;
    xy[(2 * m + 1) * N + i] = sy;
    z[e] = init_sz;
}

// Noise of step t (read from the device counter): eta^{x,y}_i for i < N into
// rows 2m, 2m+1 of eta; the collective pair for i = N into xi[m].
__global__ void k_noise_f64(double* eta, double* xi, int64_t M, int64_t N, uint64_t seed, const int64_t* d_t,
                            int64_t m0) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t NP = N + 1;
    if (e >= M * NP) return;
    const int64_t m = e / NP, i = e - m * NP;
    const uint32_t t = (uint32_t)(*d_t);
    double gx, gy;
    normal2_f64(seed, (uint32_t)(m0 + m), t, (uint32_t)i, gx, gy);
    if (i < N) {
        eta[(2 * m) * N + i] = gx;
        eta[(2 * m + 1) * N + i] = gy;
    } else {
        xi[2 * m] = gx;
        xi[2 * m + 1] = gy;
    }
}

// Collective sums S^a = sum_i s^a_i, one warp per trajectory.
__global__ void k_sums_f64(const double* xy, const double* z, double* S, int64_t M, int64_t N) {
    const int64_t m = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (m >= M) return;
    double sx = 0, sy = 0, sz = 0;
    for (int64_t i = lane; i < N; i += 32) {
        sx += xy[(2 * m) * N + i];
        sy += xy[(2 * m + 1) * N + i];
        sz += z[m * N + i];
    }
    for (int o = 16; o; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    if (lane == 0) {
        S[4 * m] = sx;
        S[4 * m + 1] = sy;
        S[4 * m + 2] = sz;
    }
}

// Heun predictor. Field increment B^a_i = 1/2 (Gamma S^a - P^a_i) dt + bn^a_i with
// the noise part bn^a_i = sqrt(Gamma dt) xi^a - sqrt(dt) (L eta^a)_i (written
// back over the L.eta buffer for the corrector). Increment f = s x (B^y, -B^x, 0)
// = (z B^x, z B^y, -(x B^x + y B^y)); predictor s~ = s + f, h = s + f/2.
__global__ void k_predict_f64(const double* xy, const double* z, const double* pf, double* q, const double* xi,
                              const double* S, double* xyp, double* zp, double* hxy, double* hz, int64_t M,
                              int64_t N, double G, double dt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N;
    const int64_t rx = (2 * m) * N + i, ry = rx + N;
    const double sg = sqrt(G * dt), sd = sqrt(dt);
    const double x = xy[rx], y = xy[ry], zz = z[e];
    const double bnx = sg * xi[2 * m] - sd * q[rx];
    const double bny = sg * xi[2 * m + 1] - sd * q[ry];
    const double Bx = 0.5 * (G * S[4 * m] - pf[rx]) * dt + bnx;
    const double By = 0.5 * (G * S[4 * m + 1] - pf[ry]) * dt + bny;
    const double fx = zz * Bx, fy = zz * By, fz = -(x * Bx + y * By);
    xyp[rx] = x + fx;
    xyp[ry] = y + fy;
    zp[e] = zz + fz;
    hxy[rx] = x + 0.5 * fx;
    hxy[ry] = y + 0.5 * fy;
    hz[e] = zz + 0.5 * fz;
    q[rx] = bnx;
    q[ry] = bny;
}

// Heun corrector s' = s + (f(s) + f(s~))/2 = h + f(s~)/2 with the same noise,
// then rescaling to |s_i| = sqrt(3). Counts non-finite results.
__global__ void k_correct_f64(const double* xyp, const double* zp, const double* pf, const double* bn,
                              const double* Sp, const double* hxy, const double* hz, double* xy, double* z,
                              int64_t M, int64_t N, double G, double dt, int renorm,
                              unsigned long long* flags) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N;
    const int64_t rx = (2 * m) * N + i, ry = rx + N;
    const double x = xyp[rx], y = xyp[ry], zz = zp[e];
    const double Bx = 0.5 * (G * Sp[4 * m] - pf[rx]) * dt + bn[rx];
    const double By = 0.5 * (G * Sp[4 * m + 1] - pf[ry]) * dt + bn[ry];
    double nx = hxy[rx] + 0.5 * (zz * Bx);
    double ny = hxy[ry] + 0.5 * (zz * By);
    double nz = hz[e] - 0.5 * (x * Bx + y * By);
    if (renorm) {
        const double s = sqrt(3.0) / sqrt(nx * nx + ny * ny + nz * nz);
        nx *= s;
        ny *= s;
        nz *= s;
    }
    if (!isfinite(nx) || !isfinite(ny) || !isfinite(nz)) atomicAdd(&flags[FLAG_NONFINITE], 1ull);
    xy[rx] = nx;
    xy[ry] = ny;
    z[e] = nz;
}

// Midpoint m = (s + s')/2 of the implicit-midpoint rotation s' = s + m x b with
// b = (B^y, -B^x, 0) (Mentink et al. 2010): with c = b/2, m - m x c = s gives
// m = (s + s x c + (s.c) c) / (1 + |c|^2), where s x c = (z B^x, z B^y,
// -(x B^x + y B^y)) / 2 and s.c = (x B^y - y B^x) / 2.
__device__ __forceinline__ void mid_rotation_f64(double x, double y, double z, double Bx, double By, double& mx,
                                                 double& my, double& mz) {
    const double hx = 0.5 * Bx, hy = 0.5 * By;
    const double sc = x * hy - y * hx;
    const double inv = 1.0 / (1.0 + hx * hx + hy * hy);
    mx = (x + z * hx + sc * hy) * inv;
    my = (y + z * hy - sc * hx) * inv;
    mz = (z - (x * hx + y * hy)) * inv;
}

// Midpoint-scheme predictor: the same field increment as k_predict_f64; writes
// the midpoint state (s + s~)/2 of the predictor rotation (the corrector's field
// is evaluated there) and the noise part over the L.eta buffer.
__global__ void k_predict_mid_f64(const double* xy, const double* z, const double* pf, double* q, const double* xi,
                                  const double* S, double* xym, double* zm, int64_t M, int64_t N, double G,
                                  double dt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N;
    const int64_t rx = (2 * m) * N + i, ry = rx + N;
    const double sg = sqrt(G * dt), sd = sqrt(dt);
    const double x = xy[rx], y = xy[ry], zz = z[e];
    const double bnx = sg * xi[2 * m] - sd * q[rx];
    const double bny = sg * xi[2 * m + 1] - sd * q[ry];
    const double Bx = 0.5 * (G * S[4 * m] - pf[rx]) * dt + bnx;
    const double By = 0.5 * (G * S[4 * m + 1] - pf[ry]) * dt + bny;
    double mx, my, mz;
    mid_rotation_f64(x, y, zz, Bx, By, mx, my, mz);
    xym[rx] = mx;
    xym[ry] = my;
    zm[e] = mz;
    q[rx] = bnx;
    q[ry] = bny;
}

// Midpoint-scheme corrector: field at the midpoint state (pf = W m, Sm its sums)
// with the same noise, s' = 2 m' - s of the rotation from s, optional rescaling
// to |s_i| = sqrt(3) (the rotation keeps it up to rounding). In place on xy, z.
__global__ void k_correct_mid_f64(const double* pf, const double* bn, const double* Sm, double* xy, double* z,
                                  int64_t M, int64_t N, double G, double dt, int renorm,
                                  unsigned long long* flags) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N;
    const int64_t rx = (2 * m) * N + i, ry = rx + N;
    const double x = xy[rx], y = xy[ry], zz = z[e];
    const double Bx = 0.5 * (G * Sm[4 * m] - pf[rx]) * dt + bn[rx];
    const double By = 0.5 * (G * Sm[4 * m + 1] - pf[ry]) * dt + bn[ry];
    double mx, my, mz;
    mid_rotation_f64(x, y, zz, Bx, By, mx, my, mz);
    double nx = 2.0 * mx - x, ny = 2.0 * my - y, nz = 2.0 * mz - zz;
    if (renorm) {
        const double s = sqrt(3.0) / sqrt(nx * nx + ny * ny + nz * nz);
        nx *= s;
        ny *= s;
        nz *= s;
    }
    if (!isfinite(nx) || !isfinite(ny) || !isfinite(nz)) atomicAdd(&flags[FLAG_NONFINITE], 1ull);
    xy[rx] = nx;
    xy[ry] = ny;
    z[e] = nz;
}

// Closing kernel of a step: collective sums of the new state, window moments
// S^z, A, A^2, A S^z, (S^z)^2 with A = ((S^x)^2 + (S^y)^2)/4 when the completed
// step count exceeds n_window, and the step counter increment by the last
// block to finish (all blocks have read the counter by then).
__global__ void k_close_f64(const double* xy, const double* z, double* S, double* mom, int64_t M, int64_t N,
                            int64_t* d_t, int64_t n_window, int64_t n_stride, int64_t* d_count,
                            unsigned long long* flags) {
    const int64_t m = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    const int64_t t1 = *d_t + 1;
    const bool sample = window_sample(t1, n_window, n_stride);
    if (m < M) {
        double sx = 0, sy = 0, sz = 0;
        for (int64_t i = lane; i < N; i += 32) {
            sx += xy[(2 * m) * N + i];
            sy += xy[(2 * m + 1) * N + i];
            sz += z[m * N + i];
        }
        for (int o = 16; o; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        }
        if (lane == 0) {
            S[4 * m] = sx;
            S[4 * m + 1] = sy;
            S[4 * m + 2] = sz;
            if (sample) {
                const double A = 0.25 * (sx * sx + sy * sy);
                double* mm = mom + 5 * m;
                mm[0] += sz;
                mm[1] += A;
                mm[2] += A * A;
                mm[3] += A * sz;
                mm[4] += sz * sz;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long done = atomicAdd(&flags[FLAG_DONE], 1ull);
        if (done == gridDim.x - 1) {
            flags[FLAG_DONE] = 0ull;
            if (sample) *d_count += 1;
            __threadfence();
            *d_t = t1;
        }
    }
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void gemm_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int64_t n_i,
              int64_t n_n, int64_t K, double alpha, double beta, bool tri_a, bool lower_only, cudaStream_t st) {
    dim3 grid(blocks_for(n_i, GT), blocks_for(n_n, GT));
    k_gemm_f64<<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, n_i, n_n, K, alpha, beta, tri_a ? 1 : 0,
                                     lower_only ? 1 : 0);
}

int f64_alloc(twa_ctx* c) {
    const size_t mn = (size_t)c->M * c->N;
    double** bufs2[] = {&c->xy, &c->xyp, &c->hxy, &c->eta, &c->pf};
    double** bufs1[] = {&c->z, &c->zp, &c->hz};
    for (auto b : bufs2)
        if (dev_malloc(c, b, sizeof(double) * 2 * mn) != cudaSuccess) return set_error(c, TWA_ENOMEM, "device state");
    for (auto b : bufs1)
        if (dev_malloc(c, b, sizeof(double) * mn) != cudaSuccess) return set_error(c, TWA_ENOMEM, "device state");
    if (dev_malloc(c, &c->xi, sizeof(double) * 2 * c->M) != cudaSuccess ||
        dev_malloc(c, &c->S, sizeof(double) * 4 * c->M) != cudaSuccess ||
        dev_malloc(c, &c->Sp, sizeof(double) * 4 * c->M) != cudaSuccess)
        return set_error(c, TWA_ENOMEM, "device state");
    return TWA_OK;
}

void f64_free(twa_ctx* c) {
    double** all[] = {&c->xy, &c->xyp, &c->hxy, &c->eta, &c->pf, &c->z, &c->zp, &c->hz, &c->xi, &c->S, &c->Sp};
    for (auto b : all) {
        dev_free(c, *b);
        *b = nullptr;
    }
}

int f64_state_changed(twa_ctx* c) {
    k_sums_f64<<<blocks_for(c->M, 8), 256, 0, c->stream>>>(c->xy, c->z, c->S, c->M, c->N);
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

int f64_init_state(twa_ctx* c) {
    k_init_f64<<<blocks_for(c->M * c->N, 256), 256, 0, c->stream>>>(c->xy, c->z, c->M, c->N, c->seed,
                                                                     (double)c->opts.init_state, c->opts.traj_offset);
    TWA_CUDA(c, cudaGetLastError());
    return f64_state_changed(c);
}

int f64_run(twa_ctx* c, int64_t steps) {
    const int64_t M = c->M, N = c->N, MN = M * N;
    cudaStream_t st = c->stream;
    const unsigned gMN = blocks_for(MN, 256);
    const int64_t m0 = c->opts.traj_offset;
    for (int64_t s = 0; s < steps; ++s) {
        {
            ProfScope p(c, TWA_PROF_NOISE);
            k_noise_f64<<<blocks_for(M * (N + 1), 256), 256, 0, st>>>(c->eta, c->xi, M, N, c->seed, c->d_t, m0);
        }
        {
            // L.eta cannot be formed in place (the GEMM reads eta), so it lands in pf first
            ProfScope p(c, TWA_PROF_GEMM64);
            gemm_f64(c->L64, N, c->eta, N, c->pf, N, N, 2 * M, N, 1.0, 0.0, true, false, st);
        }
        std::swap(c->eta, c->pf);  // eta now holds L.eta
        {
            ProfScope p(c, TWA_PROF_GEMM64);
            gemm_f64(c->W64, N, c->xy, N, c->pf, N, N, 2 * M, N, 1.0, 0.0, false, false, st);
        }
        const bool mid = c->opts.integrator == TWA_INT_MIDPOINT;
        {
            // xyp, zp: the predictor s~ (Heun) or the midpoint (s + s~)/2 (midpoint scheme)
            ProfScope p(c, TWA_PROF_ELEM64);
            if (mid)
                k_predict_mid_f64<<<gMN, 256, 0, st>>>(c->xy, c->z, c->pf, c->eta, c->xi, c->S, c->xyp, c->zp, M, N,
                                                       c->Gamma, c->dt);
            else
                k_predict_f64<<<gMN, 256, 0, st>>>(c->xy, c->z, c->pf, c->eta, c->xi, c->S, c->xyp, c->zp, c->hxy,
                                                   c->hz, M, N, c->Gamma, c->dt);
        }
        {
            ProfScope p(c, TWA_PROF_ELEM64);
            k_sums_f64<<<blocks_for(M, 8), 256, 0, st>>>(c->xyp, c->zp, c->Sp, M, N);
        }
        {
            ProfScope p(c, TWA_PROF_GEMM64);
            gemm_f64(c->W64, N, c->xyp, N, c->pf, N, N, 2 * M, N, 1.0, 0.0, false, false, st);
        }
        {
            ProfScope p(c, TWA_PROF_ELEM64);
            if (mid)
                k_correct_mid_f64<<<gMN, 256, 0, st>>>(c->pf, c->eta, c->Sp, c->xy, c->z, M, N, c->Gamma, c->dt,
                                                       c->opts.renormalize, c->d_flags);
            else
                k_correct_f64<<<gMN, 256, 0, st>>>(c->xyp, c->zp, c->pf, c->eta, c->Sp, c->hxy, c->hz, c->xy,
                                                   c->z, M, N, c->Gamma, c->dt, c->opts.renormalize, c->d_flags);
        }
        {
            ProfScope p(c, TWA_PROF_CLOSE);
            k_close_f64<<<blocks_for(M, 8), 256, 0, st>>>(c->xy, c->z, c->S, c->mom, M, N, c->d_t, c->n_window,
                                                           c->n_stride, c->d_count, c->d_flags);
        }
    }
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

int f64_field(twa_ctx* c, const double* s, double* P, int64_t K, int which) {
    // L is lower triangular: the K range of each row tile stops at its end
    gemm_f64(which == 1 ? c->L64 : c->W64, c->N, s, c->N, P, c->N, c->N, K, c->N, 1.0, 0.0, which == 1, false,
             c->stream);
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

}  // namespace twa

// Pathwise gradients of a steady-state objective with respect to the pump
// parameters w and alpha of Eq. 2, at fixed noise: reverse mode through the
// stochastic-Heun step of Eq. S1 with step checkpointing.
//
// One step (the forward below, same formulas as the FP64 path), per trajectory:
//   Q = L eta, Bn = sqrt(G dt) xi - sqrt(dt) Q,   B(s) = 1/2 (G S - W s) dt + Bn,
//   f(s, B) = (z B^x, z B^y, -(x B^x + y B^y)),    s~ = s + f(s, B(s)),
//   u = s + 1/2 (f(s, B(s)) + f(s~, B(s~))),        s' = sqrt(3) u / |u|.
// Reverse step for a cotangent lambda of s' (plus the objective's source):
//   lambda_u = sqrt(3)/|u| (lambda - (lambda.u^) u^),  mu~ = lambda_u / 2,
//   pull mu~ back through f at (s~, B~):  beta~ = (mu~x z~ - mu~z x~, mu~y z~ - mu~z y~)
//   (cotangent of B~), g~ = (-mu~z B~x, -mu~z B~y, mu~x B~x + mu~y B~y), and
//   lambda_s~ = g~ + 1/2 dt (G sum_i beta~ - W beta~) on x, y;
//   mu = lambda_u / 2 + lambda_s~ pulled back the same way through f at (s, B),
//   lambda_s = lambda_u + lambda_s~ + g + 1/2 dt (G sum_i beta - W beta).
// Parameter derivatives: dJ/dtheta += sum (beta + beta~) . dBn/dtheta
//   - 1/2 dt (beta . dW s + beta~ . dW s~), dBn/dtheta = -sqrt(dt) dL eta.
// W is symmetric, so W^T beta = W beta.
#include <math.h>

#include "twa_internal.cuh"

namespace twa {
namespace {

constexpr int AT = 256;

template <typename T>
__global__ void k_a_init(T* xy, T* z, int64_t M, int64_t N, uint64_t seed, double init_sz, int64_t m0) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N;
    double sx, sy;
    init_signs(seed, (uint32_t)(m0 + m), (uint32_t)i, sx, sy);
    xy[(2 * m) * N + i] = (T)sx;
    xy[(2 * m + 1) * N + i] = (T)sy;
    z[e] = (T)init_sz;
}

// Noise of step t, drawn exactly as the forward path of the same precision draws it.
template <typename T>
__global__ void k_a_noise(T* eta, T* xi, int64_t M, int64_t N, uint64_t seed, int64_t t, int64_t m0) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t NP = N + 1;
    if (e >= M * NP) return;
    const int64_t m = e / NP, i = e - m * NP;
    T gx, gy;
    if (sizeof(T) == 8) {
        double a, b;
        normal2_f64(seed, (uint32_t)(m0 + m), (uint32_t)t, (uint32_t)i, a, b);
        gx = (T)a;
        gy = (T)b;
    } else {
        float a, b;
        normal2_f32(seed, (uint32_t)(m0 + m), (uint32_t)t, (uint32_t)i, a, b);
        if (i < N) {   // the mixed path's pump noise is the BF16 value
            a = __bfloat162float(__float2bfloat16_rn(a));
            b = __bfloat162float(__float2bfloat16_rn(b));
        }
        gx = (T)a;
        gy = (T)b;
    }
    if (i < N) {
        eta[(2 * m) * N + i] = gx;
        eta[(2 * m + 1) * N + i] = gy;
    } else {
        xi[2 * m] = gx;
        xi[2 * m + 1] = gy;
    }
}

// Collective sums S = (sum x, sum y, sum z) in FP64, one warp per trajectory.
template <typename T>
__global__ void k_a_sums(const T* xy, const T* z, double* S, int64_t M, int64_t N) {
    const int64_t m = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (m >= M) return;
    double sx = 0, sy = 0, sz = 0;
    for (int64_t i = lane; i < N; i += 32) {
        sx += (double)xy[(2 * m) * N + i];
        sy += (double)xy[(2 * m + 1) * N + i];
        sz += (double)z[m * N + i];
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

template <typename T>
struct Field {   // B(s) at one site: 1/2 (G S - P) dt + Bn
    T bx, by;
};

template <typename T>
__device__ __forceinline__ Field<T> field_at(const double* S, int64_t m, T Px, T Py, T Qx, T Qy, const T* xi, T G,
                                             T dt, T sg, T sd) {
    Field<T> f;
    f.bx = (T)0.5 * (G * (T)S[4 * m] - Px) * dt + (sg * xi[2 * m] - sd * Qx);
    f.by = (T)0.5 * (G * (T)S[4 * m + 1] - Py) * dt + (sg * xi[2 * m + 1] - sd * Qy);
    return f;
}

template <typename T>
__global__ void k_a_pred(const T* xy, const T* z, const T* P, const T* Q, const T* xi, const double* S, T* xyt, T* zt,
                         int64_t M, int64_t N, T G, T dt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N, rx = (2 * m) * N + i, ry = rx + N;
    const T sg = sqrt(G * dt), sd = sqrt(dt);
    const T x = xy[rx], y = xy[ry], zz = z[e];
    const Field<T> B = field_at<T>(S, m, P[rx], P[ry], Q[rx], Q[ry], xi, G, dt, sg, sd);
    xyt[rx] = x + zz * B.bx;
    xyt[ry] = y + zz * B.by;
    zt[e] = zz - (x * B.bx + y * B.by);
}

template <typename T>
__global__ void k_a_corr(const T* xy, const T* z, const T* xyt, const T* zt, const T* P, const T* Pt, const T* Q,
                         const T* xi, const double* S, const double* St, T* xyn, T* zn, int64_t M, int64_t N, T G, T dt,
                         int renorm, unsigned long long* flags) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N, rx = (2 * m) * N + i, ry = rx + N;
    const T sg = sqrt(G * dt), sd = sqrt(dt);
    const T x = xy[rx], y = xy[ry], zz = z[e];
    const T xt = xyt[rx], yt = xyt[ry], ztt = zt[e];
    const Field<T> B = field_at<T>(S, m, P[rx], P[ry], Q[rx], Q[ry], xi, G, dt, sg, sd);
    const Field<T> Bt = field_at<T>(St, m, Pt[rx], Pt[ry], Q[rx], Q[ry], xi, G, dt, sg, sd);
    T ux = x + (T)0.5 * (zz * B.bx + ztt * Bt.bx);
    T uy = y + (T)0.5 * (zz * B.by + ztt * Bt.by);
    T uz = zz - (T)0.5 * (x * B.bx + y * B.by + xt * Bt.bx + yt * Bt.by);
    if (renorm) {
        const T s = sqrt((T)3 / (ux * ux + uy * uy + uz * uz));
        ux *= s;
        uy *= s;
        uz *= s;
    }
    if (!(isfinite((double)ux) && isfinite((double)uy) && isfinite((double)uz))) atomicAdd(&flags[FLAG_NONFINITE], 1ull);
    xyn[rx] = ux;
    xyn[ry] = uy;
    zn[e] = uz;
}

// Window moments of the forward run: phi(S) = (S^z, A, A^2, A S^z, (S^z)^2).
__global__ void k_a_moments(const double* S, double* mom, int64_t M) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double sx = S[4 * m], sy = S[4 * m + 1], sz = S[4 * m + 2];
    const double A = 0.25 * (sx * sx + sy * sy);
    double* mm = mom + 5 * m;
    mm[0] += sz;
    mm[1] += A;
    mm[2] += A * A;
    mm[3] += A * sz;
    mm[4] += sz * sz;
}

// Ensemble means -> objective J and its coefficients c (J ~ sum_k c_k mu_k to
// first order); out = c[0..4], J, scale = 1 / (M samples).
__global__ void k_a_objective(const double* mom, int64_t M, int64_t nsamp, int objective, double* out) {
    __shared__ double sm[5][256];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x)
        for (int k = 0; k < 5; ++k) acc[k] += mom[5 * m + k];
    for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double mu[5];
    for (int k = 0; k < 5; ++k) mu[k] = sm[k][0] / ((double)M * (double)nsamp);
    const double spsm = mu[1] + 0.5 * mu[0];
    const double dsp[5] = {0.5, 1.0, 0.0, 0.0, 0.0};
    double c[5], J;
    if (objective == TWA_OBJ_SPSM) {
        for (int k = 0; k < 5; ++k) c[k] = dsp[k];
        J = spsm;
    } else {
        const double g2n = mu[2] + 2.0 * mu[3] - mu[0] / 3.0 + 0.5 * mu[4] - 4.0 / 3.0 * mu[1];
        const double dg[5] = {-1.0 / 3.0, -4.0 / 3.0, 1.0, 2.0, 0.5};
        for (int k = 0; k < 5; ++k) c[k] = dg[k] / (spsm * spsm) - 2.0 * g2n / (spsm * spsm * spsm) * dsp[k];
        J = g2n / (spsm * spsm);
    }
    for (int k = 0; k < 5; ++k) out[k] = c[k];
    out[5] = J;
    out[6] = 1.0 / ((double)M * (double)nsamp);
    for (int k = 0; k < 5; ++k) out[7 + k] = mu[k];
}

template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T* sm) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    T t = (l < AT / 32) ? sm[l] : (T)0;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// Reverse step, part 1: objective source, renormalisation and the pull-back of
// lambda_u / 2 through f at (s~, B~). Grid (ceil(N / AT), M).
template <typename T>
__global__ void k_b1(const T* lxy, const T* lz, const T* xy, const T* z, const T* xyt, const T* zt, const T* P,
                     const T* Pt, const T* Q, const T* xi, const double* S, const double* St, const double* Sn,
                     const double* obj, int in_window, T* luxy, T* luz, T* btxy, T* gtxy, T* gtz, double* sumbt,
                     int64_t M, int64_t N, T G, T dt, int renorm) {
    __shared__ T sm[32];
    const int64_t m = blockIdx.y, i = blockIdx.x * (int64_t)AT + threadIdx.x;
    const bool ok = i < N;
    T bx = 0, by = 0;
    if (ok) {
        const int64_t e = m * N + i, rx = (2 * m) * N + i, ry = rx + N;
        const T sg = sqrt(G * dt), sd = sqrt(dt);
        T l0 = lxy[rx], l1 = lxy[ry], l2 = lz[e];
        if (in_window) {
            // d J / d s^a_i = scale sum_k c_k d phi_k / d S^a at the state after this step
            const double Sx = Sn[4 * m], Sy = Sn[4 * m + 1], Sz = Sn[4 * m + 2];
            const double A = 0.25 * (Sx * Sx + Sy * Sy), sc = obj[6];
            const double gx = 0.5 * Sx * (obj[1] + 2.0 * A * obj[2] + Sz * obj[3]);
            const double gy = 0.5 * Sy * (obj[1] + 2.0 * A * obj[2] + Sz * obj[3]);
            const double gz = obj[0] + A * obj[3] + 2.0 * Sz * obj[4];
            l0 += (T)(sc * gx);
            l1 += (T)(sc * gy);
            l2 += (T)(sc * gz);
        }
        const T x = xy[rx], y = xy[ry], zz = z[e];
        const T xt = xyt[rx], yt = xyt[ry], ztt = zt[e];
        const Field<T> B = field_at<T>(S, m, P[rx], P[ry], Q[rx], Q[ry], xi, G, dt, sg, sd);
        const Field<T> Bt = field_at<T>(St, m, Pt[rx], Pt[ry], Q[rx], Q[ry], xi, G, dt, sg, sd);
        if (renorm) {
            const T ux = x + (T)0.5 * (zz * B.bx + ztt * Bt.bx);
            const T uy = y + (T)0.5 * (zz * B.by + ztt * Bt.by);
            const T uz = zz - (T)0.5 * (x * B.bx + y * B.by + xt * Bt.bx + yt * Bt.by);
            const T n = sqrt(ux * ux + uy * uy + uz * uz), inv = (T)1 / n;
            const T dot = (l0 * ux + l1 * uy + l2 * uz) * inv;
            const T k = sqrt((T)3) * inv;
            l0 = k * (l0 - dot * ux * inv);
            l1 = k * (l1 - dot * uy * inv);
            l2 = k * (l2 - dot * uz * inv);
        }
        luxy[rx] = l0;
        luxy[ry] = l1;
        luz[e] = l2;
        const T mx = (T)0.5 * l0, my = (T)0.5 * l1, mz = (T)0.5 * l2;
        bx = mx * ztt - mz * xt;
        by = my * ztt - mz * yt;
        btxy[rx] = bx;
        btxy[ry] = by;
        gtxy[rx] = -mz * Bt.bx;
        gtxy[ry] = -mz * Bt.by;
        gtz[e] = mx * Bt.bx + my * Bt.by;
    }
    const T sx = block_sum_t<T>(bx, sm);
    const T sy = block_sum_t<T>(by, sm);
    if (threadIdx.x == 0) {
        atomicAdd(&sumbt[2 * m], (double)sx);
        atomicAdd(&sumbt[2 * m + 1], (double)sy);
    }
}

// Reverse step, part 2: lambda_s~, the pull-back through f at (s, B), and the
// w-derivative terms (dW/dw = W/w, dL/dw = L/(2w) reuse W s, W s~, L eta).
template <typename T>
__global__ void k_b2(const T* luxy, const T* luz, const T* gtxy, const T* gtz, const T* Wbt, const double* sumbt,
                     const T* btxy, const T* xy, const T* z, const T* P, const T* Pt, const T* Q, const T* xi,
                     const double* S, T* bxy, T* lpxy, T* lpz, double* sumb, double* gpart, int64_t M, int64_t N,
                     T G, T dt, double w) {
    __shared__ T sm[32];
    const int64_t m = blockIdx.y, i = blockIdx.x * (int64_t)AT + threadIdx.x;
    const bool ok = i < N;
    T bx = 0, by = 0, gw = 0;
    if (ok) {
        const int64_t e = m * N + i, rx = (2 * m) * N + i, ry = rx + N;
        const T sg = sqrt(G * dt), sd = sqrt(dt), hd = (T)0.5 * dt;
        const T ltx = gtxy[rx] + hd * (G * (T)sumbt[2 * m] - Wbt[rx]);
        const T lty = gtxy[ry] + hd * (G * (T)sumbt[2 * m + 1] - Wbt[ry]);
        const T ltz = gtz[e];
        const T ux = luxy[rx], uy = luxy[ry], uz = luz[e];
        const T mx = (T)0.5 * ux + ltx, my = (T)0.5 * uy + lty, mz = (T)0.5 * uz + ltz;
        const T x = xy[rx], y = xy[ry], zz = z[e];
        const Field<T> B = field_at<T>(S, m, P[rx], P[ry], Q[rx], Q[ry], xi, G, dt, sg, sd);
        bx = mx * zz - mz * x;
        by = my * zz - mz * y;
        bxy[rx] = bx;
        bxy[ry] = by;
        lpxy[rx] = ux + ltx - mz * B.bx;
        lpxy[ry] = uy + lty - mz * B.by;
        lpz[e] = uz + ltz + mx * B.bx + my * B.by;
        const T btx = btxy[rx], bty = btxy[ry];
        gw = -hd * (bx * P[rx] + by * P[ry] + btx * Pt[rx] + bty * Pt[ry]) -
             (T)0.5 * sd * ((bx + btx) * Q[rx] + (by + bty) * Q[ry]);
    }
    const T sx = block_sum_t<T>(bx, sm);
    const T sy = block_sum_t<T>(by, sm);
    const T sw = block_sum_t<T>(gw, sm);
    if (threadIdx.x == 0) {
        atomicAdd(&sumb[2 * m], (double)sx);
        atomicAdd(&sumb[2 * m + 1], (double)sy);
        atomicAdd(&gpart[2 * m], (double)sw / w);
    }
}

// Reverse step, part 3: lambda_s, and the alpha-derivative terms with
// dW/dalpha s, dW/dalpha s~ and dL/dalpha eta.
template <typename T>
__global__ void k_b3(const T* lpxy, const T* lpz, const T* Wb, const double* sumb, const T* bxy, const T* btxy,
                     const T* Ds, const T* Dst, const T* LdE, T* lxy, T* lz, double* gpart, int64_t M, int64_t N, T G,
                     T dt, int want_alpha) {
    __shared__ T sm[32];
    const int64_t m = blockIdx.y, i = blockIdx.x * (int64_t)AT + threadIdx.x;
    const bool ok = i < N;
    T ga = 0;
    if (ok) {
        const int64_t e = m * N + i, rx = (2 * m) * N + i, ry = rx + N;
        const T hd = (T)0.5 * dt, sd = sqrt(dt);
        lxy[rx] = lpxy[rx] + hd * (G * (T)sumb[2 * m] - Wb[rx]);
        lxy[ry] = lpxy[ry] + hd * (G * (T)sumb[2 * m + 1] - Wb[ry]);
        lz[e] = lpz[e];
        if (want_alpha) {
            const T bx = bxy[rx], by = bxy[ry], btx = btxy[rx], bty = btxy[ry];
            ga = -hd * (bx * Ds[rx] + by * Ds[ry] + btx * Dst[rx] + bty * Dst[ry]) -
                 sd * ((bx + btx) * LdE[rx] + (by + bty) * LdE[ry]);
        }
    }
    if (want_alpha) {
        const T sa = block_sum_t<T>(ga, sm);
        if (threadIdx.x == 0) atomicAdd(&gpart[2 * m + 1], (double)sa);
    }
}

// Per-trajectory samples M * gpart, their means and standard errors.
__global__ void k_a_reduce(const double* gpart, int64_t M, double* out) {
    __shared__ double sm[4][256];
    double a[4] = {0, 0, 0, 0};
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x) {
        const double g0 = M * gpart[2 * m], g1 = M * gpart[2 * m + 1];
        a[0] += g0;
        a[1] += g0 * g0;
        a[2] += g1;
        a[3] += g1 * g1;
    }
    for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int p = 0; p < 2; ++p) {
            const double mean = sm[2 * p][0] / M;
            const double var = (M > 1) ? (sm[2 * p + 1][0] - M * mean * mean) / (M - 1) : 0.0;
            out[2 * p] = mean;
            out[2 * p + 1] = (M > 1) ? sqrt(fmax(var, 0.0) / M) : NAN;
        }
    }
}

__global__ void k_a_scale_copy(const double* gpart, double* out, int64_t M) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < 2 * M) out[e] = (double)M * gpart[e];
}

// dW/dalpha = -ln(1 + |i - j|) W_ij.
__global__ void k_a_dalpha(const double* W, double* D, int64_t N) {
    const int64_t n2 = N * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N, j = e - i * N;
        const int64_t d = i > j ? i - j : j - i;
        D[e] = -log1p((double)d) * W[e];
    }
}

__global__ void k_a_transpose(const double* A, double* B, int64_t N) {
    __shared__ double t[32][33];
    const int64_t bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = by + k, cidx = bx + threadIdx.x;
        if (r < N && cidx < N) t[k][threadIdx.x] = A[r * N + cidx];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = bx + k, cidx = by + threadIdx.x;
        if (r < N && cidx < N) B[r * N + cidx] = t[threadIdx.x][k];
    }
}

// In the diagonal block [k0, k0 + kb) of every row c of Y (= X^T): solve
// L_kk y = y (forward substitution), the block's rows of X = L^-1 B.
__global__ void k_a_trsm_block(const double* L, double* Y, int64_t N, int64_t k0, int kb) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    double y[32];
    for (int r = 0; r < kb; ++r) {
        double v = Y[c * N + k0 + r];
        for (int q = 0; q < r; ++q) v -= L[(k0 + r) * N + k0 + q] * y[q];
        y[r] = v / L[(k0 + r) * N + k0 + r];
    }
    for (int r = 0; r < kb; ++r) Y[c * N + k0 + r] = y[r];
}

// B[j][k] = Phi(X)[k][j]: lower triangle of X with the diagonal halved, transposed.
__global__ void k_a_phi_t(const double* X, double* B, int64_t N) {
    const int64_t n2 = N * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / N, k = e - j * N;
        B[e] = (k > j) ? X[k * N + j] : (k == j ? 0.5 * X[k * N + k] : 0.0);
    }
}

inline unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Y <- (L^-1 Y^T)^T in place: blocked forward substitution on the transposed
// right-hand sides, with the FP64 GEMM for the off-diagonal updates.
int trsm_lower_t(twa_ctx* c, double* Y) {
    const int64_t N = c->N;
    for (int64_t k0 = 0; k0 < N; k0 += 32) {
        const int kb = (int)((N - k0) < 32 ? (N - k0) : 32);
        if (k0 > 0)
            gemm_f64(c->L64 + k0 * N, N, Y, N, Y + k0, N, kb, N, k0, -1.0, 1.0, false, false, c->stream);
        k_a_trsm_block<<<nb(N, 128), 128, 0, c->stream>>>(c->L64, Y, N, k0, kb);
    }
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

// dL/dalpha = L Phi(L^-1 D L^-T) (Cholesky derivative), FP64.
int factor_derivative(twa_ctx* c, const double* D, double* Ld, double* tmp) {
    const int64_t N = c->N;
    const dim3 tb(32, 8), tg(nb(N, 32), nb(N, 32));
    TWA_CUDA(c, cudaMemcpyAsync(tmp, D, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c->stream));
    int rc;
    if ((rc = trsm_lower_t(c, tmp))) return rc;          // tmp = (L^-1 D)^T
    k_a_transpose<<<tg, tb, 0, c->stream>>>(tmp, Ld, N);  // Ld = L^-1 D
    if ((rc = trsm_lower_t(c, Ld))) return rc;           // Ld = (L^-1 (L^-1 D)^T)^T = L^-1 D L^-T (symmetric)
    k_a_phi_t<<<4096, 256, 0, c->stream>>>(Ld, tmp, N);   // tmp[j][k] = Phi[k][j]
    gemm_f64(c->L64, N, tmp, N, Ld, N, N, N, N, 1.0, 0.0, false, false, c->stream);   // Ld[j][i] = (L Phi)[i][j]
    k_a_transpose<<<tg, tb, 0, c->stream>>>(Ld, tmp, N);
    TWA_CUDA(c, cudaMemcpyAsync(Ld, tmp, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c->stream));
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

template <typename T>
struct Adjoint {
    twa_ctx* c;
    int64_t M, N, C, steps, nck, nsamp;
    bool want_alpha;
    double* D64 = nullptr;     // dW/dalpha
    double* Ld64 = nullptr;    // dL/dalpha
    std::vector<void*> owned;
    // state, checkpoints, tape
    T *xy, *z, *xy2, *z2, *ck, *eta, *xiS;
    T *txy, *tz, *ttxy, *ttz, *tP, *tPt, *tQ, *txi;
    double *tS, *tSt, *tSn, *mom, *obj, *gpart, *sumbt, *sumb, *res;
    T *lxy, *lz, *luxy, *luz, *btxy, *gtxy, *gtz, *Wbt, *bxy, *lpxy, *lpz, *Wb, *Ds, *Dst, *LdE;

    template <typename U>
    int alloc(U** p, size_t n) {
        if (dev_malloc(c, p, sizeof(U) * n) != cudaSuccess) return set_error(c, TWA_ENOMEM, "twa_grad: device allocation");
        owned.push_back(*p);
        return TWA_OK;
    }
    ~Adjoint() {
        cudaStreamSynchronize(c->stream);
        for (void* p : owned) dev_free(c, p);
    }

    int contract(int which, const T* in, T* out) {
        if (sizeof(T) == 8) {
            const double* A = which == 0 ? c->W64 : which == 1 ? c->L64 : which == 2 ? D64 : Ld64;
            gemm_f64(A, N, (const double*)in, N, (double*)out, N, N, 2 * M, N, 1.0, 0.0, which == 1 || which == 3,
                     false, c->stream);
            TWA_CUDA(c, cudaGetLastError());
            return TWA_OK;
        }
        return tc_contract_f32(c, which, (const float*)in, (float*)out, 2 * M);
    }

    int setup() {
        const size_t MN = (size_t)M * N;
        int rc;
        if ((rc = alloc(&xy, 2 * MN)) || (rc = alloc(&z, MN)) || (rc = alloc(&xy2, 2 * MN)) || (rc = alloc(&z2, MN)) ||
            (rc = alloc(&ck, 3 * MN * nck)) || (rc = alloc(&eta, 2 * MN)) || (rc = alloc(&xiS, 2 * M)))
            return rc;
        if ((rc = alloc(&txy, 2 * MN * C)) || (rc = alloc(&tz, MN * C)) || (rc = alloc(&ttxy, 2 * MN * C)) ||
            (rc = alloc(&ttz, MN * C)) || (rc = alloc(&tP, 2 * MN * C)) || (rc = alloc(&tPt, 2 * MN * C)) ||
            (rc = alloc(&tQ, 2 * MN * C)) || (rc = alloc(&txi, 2 * M * C)))
            return rc;
        if ((rc = alloc(&tS, 4 * M * C)) || (rc = alloc(&tSt, 4 * M * C)) || (rc = alloc(&tSn, 4 * M * C)) ||
            (rc = alloc(&mom, 5 * M)) || (rc = alloc(&obj, 16)) || (rc = alloc(&gpart, 2 * M)) ||
            (rc = alloc(&sumbt, 2 * M)) || (rc = alloc(&sumb, 2 * M)) || (rc = alloc(&res, 8)))
            return rc;
        T** vec2[] = {&lxy, &luxy, &btxy, &gtxy, &Wbt, &bxy, &lpxy, &Wb, &Ds, &Dst, &LdE};
        for (auto p : vec2)
            if ((rc = alloc(p, 2 * MN))) return rc;
        T** vec1[] = {&lz, &luz, &gtz, &lpz};
        for (auto p : vec1)
            if ((rc = alloc(p, MN))) return rc;
        TWA_CUDA(c, cudaMemsetAsync(mom, 0, sizeof(double) * 5 * M, c->stream));
        TWA_CUDA(c, cudaMemsetAsync(gpart, 0, sizeof(double) * 2 * M, c->stream));
        if (want_alpha) {
            double* tmp = nullptr;
            if ((rc = alloc(&D64, (size_t)N * N)) || (rc = alloc(&Ld64, (size_t)N * N)) ||
                (rc = alloc(&tmp, (size_t)N * N)))
                return rc;
            k_a_dalpha<<<4096, 256, 0, c->stream>>>(c->W64, D64, N);
            if ((rc = factor_derivative(c, D64, Ld64, tmp))) return rc;
            if (sizeof(T) == 4) {
                if ((rc = tc_set_extra_matrix(c, 0, D64)) || (rc = tc_set_extra_matrix(c, 1, Ld64))) return rc;
            }
        }
        return TWA_OK;
    }

    // One forward step from (sxy, sz) into (nxy, nz), recording into tape slot k.
    int step(int64_t t, const T* sxy, const T* sz, T* nxy, T* nz, int64_t k) {
        const size_t MN = (size_t)M * N;
        T *sxt = ttxy + 2 * MN * k, *szt = ttz + MN * k, *P = tP + 2 * MN * k, *Pt = tPt + 2 * MN * k;
        T *Q = tQ + 2 * MN * k, *xi = txi + 2 * M * k;
        double *S = tS + 4 * M * k, *St = tSt + 4 * M * k, *Sn = tSn + 4 * M * k;
        const T G = (T)c->Gamma, dt = (T)c->dt;
        int rc;
        k_a_noise<T><<<nb(M * (N + 1), AT), AT, 0, c->stream>>>(eta, xi, M, N, c->seed, t, c->opts.traj_offset);
        if ((rc = contract(1, eta, Q))) return rc;
        k_a_sums<T><<<nb(M, 8), 256, 0, c->stream>>>(sxy, sz, S, M, N);
        if ((rc = contract(0, sxy, P))) return rc;
        k_a_pred<T><<<nb(MN, AT), AT, 0, c->stream>>>(sxy, sz, P, Q, xi, S, sxt, szt, M, N, G, dt);
        k_a_sums<T><<<nb(M, 8), 256, 0, c->stream>>>(sxt, szt, St, M, N);
        if ((rc = contract(0, sxt, Pt))) return rc;
        k_a_corr<T><<<nb(MN, AT), AT, 0, c->stream>>>(sxy, sz, sxt, szt, P, Pt, Q, xi, S, St, nxy, nz, M, N, G, dt,
                                                      c->opts.renormalize, c->d_flags);
        k_a_sums<T><<<nb(M, 8), 256, 0, c->stream>>>(nxy, nz, Sn, M, N);
        TWA_CUDA(c, cudaGetLastError());
        return TWA_OK;
    }

    int forward() {
        const size_t MN = (size_t)M * N;
        k_a_init<T><<<nb(MN, AT), AT, 0, c->stream>>>(xy, z, M, N, c->seed, (double)c->opts.init_state,
                                                      c->opts.traj_offset);
        T *a = xy, *az = z, *b = xy2, *bz = z2;
        for (int64_t t = 0; t < steps; ++t) {
            if (t % C == 0) {
                T* dst = ck + 3 * MN * (t / C);
                TWA_CUDA(c, cudaMemcpyAsync(dst, a, sizeof(T) * 2 * MN, cudaMemcpyDeviceToDevice, c->stream));
                TWA_CUDA(c, cudaMemcpyAsync(dst + 2 * MN, az, sizeof(T) * MN, cudaMemcpyDeviceToDevice, c->stream));
            }
            int rc;
            if ((rc = step(t, a, az, b, bz, 0))) return rc;
            if (window_sample(t + 1, c->n_window, c->n_stride))
                k_a_moments<<<nb(M, 256), 256, 0, c->stream>>>(tSn, mom, M);
            std::swap(a, b);
            std::swap(az, bz);
        }
        return TWA_OK;
    }

    int backward() {
        const size_t MN = (size_t)M * N;
        const T G = (T)c->Gamma, dt = (T)c->dt;
        TWA_CUDA(c, cudaMemsetAsync(lxy, 0, sizeof(T) * 2 * MN, c->stream));
        TWA_CUDA(c, cudaMemsetAsync(lz, 0, sizeof(T) * MN, c->stream));
        const dim3 g2(nb(N, AT), (unsigned)M);
        for (int64_t blk = nck - 1; blk >= 0; --blk) {
            const int64_t t0 = blk * C, t1 = (t0 + C < steps) ? t0 + C : steps;
            // recompute the block, keeping every step's inputs on the tape
            T* src = ck + 3 * MN * blk;
            TWA_CUDA(c, cudaMemcpyAsync(txy, src, sizeof(T) * 2 * MN, cudaMemcpyDeviceToDevice, c->stream));
            TWA_CUDA(c, cudaMemcpyAsync(tz, src + 2 * MN, sizeof(T) * MN, cudaMemcpyDeviceToDevice, c->stream));
            int rc;
            for (int64_t t = t0; t < t1; ++t) {
                const int64_t k = t - t0;
                T* nxy = (k + 1 < C) ? txy + 2 * MN * (k + 1) : xy2;
                T* nz = (k + 1 < C) ? tz + MN * (k + 1) : z2;
                if ((rc = step(t, txy + 2 * MN * k, tz + MN * k, nxy, nz, k))) return rc;
            }
            for (int64_t t = t1 - 1; t >= t0; --t) {
                const int64_t k = t - t0;
                const T *sxy = txy + 2 * MN * k, *sz = tz + MN * k, *sxt = ttxy + 2 * MN * k, *szt = ttz + MN * k;
                const T *P = tP + 2 * MN * k, *Pt = tPt + 2 * MN * k, *Q = tQ + 2 * MN * k, *xi = txi + 2 * M * k;
                const double *S = tS + 4 * M * k, *St = tSt + 4 * M * k, *Sn = tSn + 4 * M * k;
                TWA_CUDA(c, cudaMemsetAsync(sumbt, 0, sizeof(double) * 2 * M, c->stream));
                TWA_CUDA(c, cudaMemsetAsync(sumb, 0, sizeof(double) * 2 * M, c->stream));
                k_b1<T><<<g2, AT, 0, c->stream>>>(lxy, lz, sxy, sz, sxt, szt, P, Pt, Q, xi, S, St, Sn, obj,
                                                  window_sample(t + 1, c->n_window, c->n_stride) ? 1 : 0, luxy, luz,
                                                  btxy, gtxy, gtz, sumbt, M, N, G, dt, c->opts.renormalize);
                if ((rc = contract(0, btxy, Wbt))) return rc;
                k_b2<T><<<g2, AT, 0, c->stream>>>(luxy, luz, gtxy, gtz, Wbt, sumbt, btxy, sxy, sz, P, Pt, Q, xi, S,
                                                  bxy, lpxy, lpz, sumb, gpart, M, N, G, dt, c->w);
                if ((rc = contract(0, bxy, Wb))) return rc;
                if (want_alpha) {
                    k_a_noise<T><<<nb(M * (N + 1), AT), AT, 0, c->stream>>>(eta, xiS, M, N, c->seed, t,
                                                                            c->opts.traj_offset);
                    if ((rc = contract(3, eta, LdE)) || (rc = contract(2, sxy, Ds)) || (rc = contract(2, sxt, Dst)))
                        return rc;
                }
                k_b3<T><<<g2, AT, 0, c->stream>>>(lpxy, lpz, Wb, sumb, bxy, btxy, Ds, Dst, LdE, lxy, lz, gpart, M, N,
                                                  G, dt, want_alpha ? 1 : 0);
                TWA_CUDA(c, cudaGetLastError());
            }
        }
        return TWA_OK;
    }
};

template <typename T>
int run_grad(twa_ctx* c, const twa_grad_req* r, twa_grad_out* out, double* per_traj) {
    Adjoint<T> a{};
    a.c = c;
    a.M = r->M;
    a.N = c->N;
    a.steps = r->steps;
    a.C = r->checkpoint > 0 ? r->checkpoint : 64;
    if (a.C > a.steps) a.C = a.steps;
    a.nck = (a.steps + a.C - 1) / a.C;
    a.nsamp = a.steps > c->n_window ? (a.steps - c->n_window) / c->n_stride : 0;
    a.want_alpha = r->want_alpha != 0;
    if (a.nsamp < 1) return set_error(c, TWA_ESTATE, "twa_grad: no step inside the averaging window");
    int rc;
    if ((rc = a.setup())) return rc;
    if ((rc = a.forward())) return rc;
    k_a_objective<<<1, 256, 0, c->stream>>>(a.mom, a.M, a.nsamp, r->objective, a.obj);
    if ((rc = a.backward())) return rc;
    k_a_reduce<<<1, 256, 0, c->stream>>>(a.gpart, a.M, a.res);
    TWA_CUDA(c, cudaGetLastError());
    double res[4], obj[16];
    TWA_CUDA(c, cudaMemcpyAsync(res, a.res, sizeof(res), cudaMemcpyDeviceToHost, c->stream));
    TWA_CUDA(c, cudaMemcpyAsync(obj, a.obj, sizeof(obj), cudaMemcpyDeviceToHost, c->stream));
    if (per_traj) {
        double* d = nullptr;
        if ((rc = a.alloc(&d, 2 * a.M))) return rc;
        k_a_scale_copy<<<nb(2 * a.M, 256), 256, 0, c->stream>>>(a.gpart, d, a.M);
        TWA_CUDA(c, cudaMemcpyAsync(per_traj, d, sizeof(double) * 2 * a.M, cudaMemcpyDeviceToHost, c->stream));
    }
    TWA_CUDA(c, cudaStreamSynchronize(c->stream));
    out->J = obj[5];
    out->dJ_dw = res[0];
    out->dJ_dw_se = res[1];
    out->dJ_dalpha = a.want_alpha ? res[2] : 0.0;
    out->dJ_dalpha_se = a.want_alpha ? res[3] : 0.0;
    out->M = a.M;
    out->steps = a.steps;
    out->samples = a.nsamp;
    for (int k = 0; k < 5; ++k) out->mu[k] = obj[7 + k];
    return TWA_OK;
}

}  // namespace

int grad(twa_ctx* c, const twa_grad_req* r, twa_grad_out* out, double* per_traj) {
    if (c->opts.precision == TWA_PREC_FP64) return run_grad<double>(c, r, out, per_traj);
    return run_grad<float>(c, r, out, per_traj);
}

}  // namespace twa

// Two-time correlation <S+(tau) S-(0)>, its spectrum S(omega) and the linewidth
// (twa_correlation): the procedure of Sec. S1 (closing part) and the linewidth
// definition of the main text ("Observables and method").
//
// After prep_steps steps of M trajectories (context A), two more copies of
// every trajectory are made (contexts B and C) with the same seed, trajectory
// indices and step counter, so all three copies draw the same noise. Copy B is
// kicked by eps delta(t) S^x, copy C by eps delta(t) S^y: every classical spin
// rotated about that axis by 2 eps (exp(i eps S^b) sigma exp(-i eps S^b) for
// Pauli spins). After every lag_stride-th step the eight per-trajectory
// quantities
//   S^x(t) S^x(t0), S^y(t) S^y(t0), S^x(t) S^y(t0), S^y(t) S^x(t0),
//   chi_xx, chi_yx, chi_xy, chi_yy     (chi_ab = (S^a of the copy kicked by S^b - S^a) / eps)
// are summed per jackknife block of trajectories. At the end, on the device:
//   C(tau) = 1/4 [(xx + yy) + i (yx - xy)] + i/8 (chi_xx + chi_yy + i chi_yx - i chi_xy),
// normalised so that tau -> 0+ gives the equal-time A + <S^z>/2 of Sec. S1
// item 6; S(omega) = 2 Re sum_k c_k e^{i omega tau_k} C(tau_k) dtau (trapezoid
// weights over the recorded lags); the FWHM of S; all again with each block
// left out (delete-one jackknife) for the standard errors.
#include <math.h>
#include <string.h>

#include <string>

#include "twa_internal.cuh"

namespace twa {
namespace {

constexpr int CORR_Q = 8;      // quantities per trajectory and lag
constexpr int CORR_JB = 32;    // jackknife blocks (at most)

// Every spin of trajectory rows [M][N] rotated by the angle 2 eps about x
// (copy B) and about y (copy C); cos and sin of 2 eps passed in FP64.
template <class T>
__global__ void k_kick(const T* xa, const T* ya, const T* za, int64_t xs, T* xb, T* yb, T* zb, T* xc, T* yc, T* zc,
                       int64_t M, int64_t N, double c2, double s2) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N;
    const int64_t o = m * xs + i, oz = m * N + i;
    const double x = xa[o], y = ya[o], z = za[oz];
    // about x: (y, z) -> (c y - s z, s y + c z)
    xb[o] = (T)x;
    yb[o] = (T)(c2 * y - s2 * z);
    zb[oz] = (T)(s2 * y + c2 * z);
    // about y: (z, x) -> (c z - s x, s z + c x)
    xc[o] = (T)(c2 * x + s2 * z);
    yc[o] = (T)y;
    zc[oz] = (T)(-s2 * x + c2 * z);
}

// Collective S^x, S^y of every trajectory of the three copies, FP64 sums of
// the state (one warp per trajectory), and the eight quantities:
// q[m] = (Xa X0, Ya Y0, Xa Y0, Ya X0, (Xb - Xa)/eps, (Yb - Ya)/eps, (Xc - Xa)/eps, (Yc - Ya)/eps).
// With `s0` NULL the sums of copy A are stored into s0w instead (the kick time t0).
struct CorrRows {
    const void *xa, *ya, *xb, *yb, *xc, *yc;
    int64_t xs;   // row stride of trajectory m (elements)
};

template <class T>
__device__ __forceinline__ double row_sum(const void* base, int64_t xs, int64_t m, int64_t N, int lane) {
    const T* r = reinterpret_cast<const T*>(base) + m * xs;
    double s = 0.0;
    for (int64_t i = lane; i < N; i += 32) s += (double)r[i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

template <class T>
__global__ void k_corr_samples(CorrRows r, int64_t M, int64_t N, const double* s0, double* s0w, double inv_eps,
                               double* q) {
    const int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (m >= M) return;   // warp-uniform
    const double Xa = row_sum<T>(r.xa, r.xs, m, N, lane), Ya = row_sum<T>(r.ya, r.xs, m, N, lane);
    if (!s0) {
        if (lane == 0) {
            s0w[2 * m] = Xa;
            s0w[2 * m + 1] = Ya;
        }
        return;
    }
    const double Xb = row_sum<T>(r.xb, r.xs, m, N, lane), Yb = row_sum<T>(r.yb, r.xs, m, N, lane);
    const double Xc = row_sum<T>(r.xc, r.xs, m, N, lane), Yc = row_sum<T>(r.yc, r.xs, m, N, lane);
    if (lane == 0) {
        const double X0 = s0[2 * m], Y0 = s0[2 * m + 1];
        double* o = q + CORR_Q * m;
        o[0] = Xa * X0;
        o[1] = Ya * Y0;
        o[2] = Xa * Y0;
        o[3] = Ya * X0;
        o[4] = (Xb - Xa) * inv_eps;
        o[5] = (Yb - Ya) * inv_eps;
        o[6] = (Xc - Xa) * inv_eps;
        o[7] = (Yc - Ya) * inv_eps;
    }
}

// Block sums of the samples of one lag: CTA b adds the trajectories
// [b M / B, (b + 1) M / B) in a fixed order into acc[b][8].
__global__ void k_corr_blocks(const double* q, int64_t M, int B, double* acc) {
    __shared__ double sm[CORR_Q][256];
    const int b = blockIdx.x;
    const int64_t lo = (int64_t)b * M / B, hi = (int64_t)(b + 1) * M / B;
    double v[CORR_Q];
    for (int k = 0; k < CORR_Q; ++k) v[k] = 0.0;
    for (int64_t m = lo + threadIdx.x; m < hi; m += blockDim.x)
        for (int k = 0; k < CORR_Q; ++k) v[k] += q[CORR_Q * m + k];
    for (int k = 0; k < CORR_Q; ++k) sm[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < CORR_Q; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < CORR_Q) acc[CORR_Q * b + threadIdx.x] = sm[threadIdx.x][0];
}

// Means of the eight quantities per lag for estimate s (s = 0: all
// trajectories; s = 1 .. B: block s - 1 left out), and C(tau) of each.
__global__ void k_corr_means(const double* acc, int64_t n_lags, int B, int64_t M, double* parts, double* C) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)(B + 1) * n_lags) return;
    const int s = (int)(e / n_lags);
    const int64_t l = e - (int64_t)s * n_lags;
    const double* a = acc + l * B * CORR_Q;
    double p[CORR_Q];
    double cnt = (double)M;
    if (s > 0) cnt -= (double)((int64_t)s * M / B - (int64_t)(s - 1) * M / B);
    for (int k = 0; k < CORR_Q; ++k) {
        double t = 0.0;
        for (int b = 0; b < B; ++b) t += a[CORR_Q * b + k];
        if (s > 0) t -= a[CORR_Q * (s - 1) + k];
        p[k] = t / cnt;
        parts[e * CORR_Q + k] = p[k];
    }
    // 1/4 [(xx + yy) + i (yx - xy)] + i/8 (chi_xx + chi_yy + i chi_yx - i chi_xy)
    C[2 * e] = 0.25 * (p[0] + p[1]) - 0.125 * (p[5] - p[6]);
    C[2 * e + 1] = 0.25 * (p[3] - p[2]) + 0.125 * (p[4] + p[7]);
}

__device__ __forceinline__ double omega_at(int64_t j, int64_t n, double omax) {
    return (j == n - 1) ? omax : -omax + (double)j * (2.0 * omax / (double)(n - 1));
}

// S_s(omega_j) = 2 Re sum_l c_l e^{i omega_j tau_l} C_s(tau_l) dtau, trapezoid weights c_l.
__global__ void k_corr_spectrum(const double* C, int64_t n_lags, int nest, int64_t n_om, double omax, double dtau,
                                double* S) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)nest * n_om) return;
    const int s = (int)(e / n_om);
    const int64_t j = e - (int64_t)s * n_om;
    const double om = omega_at(j, n_om, omax);
    const double* c = C + 2 * (int64_t)s * n_lags;
    double acc = 0.0;
    for (int64_t l = 0; l < n_lags; ++l) {
        double sn, cs;
        sincos(om * ((double)l * dtau), &sn, &cs);
        const double wgt = (n_lags > 1 && (l == 0 || l == n_lags - 1)) ? 0.5 : 1.0;
        acc += wgt * (cs * c[2 * l] - sn * c[2 * l + 1]);
    }
    S[e] = 2.0 * acc * dtau;
}

// Full width at half maximum of one spectrum: the first grid maximum, then on
// each side the first interval where S falls to half of it, crossing by linear
// interpolation (NaN when a side never falls to half).
__device__ double fwhm_of(const double* S, int64_t n, double omax, int64_t* kmax) {
    int64_t k = 0;
    for (int64_t j = 1; j < n; ++j)
        if (S[j] > S[k]) k = j;
    *kmax = k;
    const double half = 0.5 * S[k];
    double left = NAN, right = NAN;
    for (int64_t j = k; j > 0; --j) {
        if (S[j - 1] <= half) {
            const double o0 = omega_at(j - 1, n, omax), o1 = omega_at(j, n, omax);
            left = o0 + (half - S[j - 1]) / (S[j] - S[j - 1]) * (o1 - o0);
            break;
        }
    }
    for (int64_t j = k; j < n - 1; ++j) {
        if (S[j + 1] <= half) {
            const double o0 = omega_at(j, n, omax), o1 = omega_at(j + 1, n, omax);
            right = o0 + (S[j] - half) / (S[j] - S[j + 1]) * (o1 - o0);
            break;
        }
    }
    return right - left;
}

// out: fwhm, fwhm_se, omega_peak, S_peak; one thread per estimate, then thread 0.
__global__ void k_corr_width(const double* S, int nest, int64_t n_om, double omax, double* out) {
    __shared__ double wd[CORR_JB + 1];
    __shared__ int64_t kk[CORR_JB + 1];
    const int s = threadIdx.x;
    if (s < nest) {
        int64_t k;
        wd[s] = fwhm_of(S + (int64_t)s * n_om, n_om, omax, &k);
        kk[s] = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int B = nest - 1;
        out[0] = wd[0];
        double se = NAN;
        if (B >= 2) {
            double mean = 0.0;
            for (int b = 1; b <= B; ++b) mean += wd[b];
            mean /= B;
            double v = 0.0;
            for (int b = 1; b <= B; ++b) v += (wd[b] - mean) * (wd[b] - mean);
            se = sqrt((double)(B - 1) / B * v);
        }
        out[1] = se;
        out[2] = omega_at(kk[0], n_om, omax);
        out[3] = S[kk[0]];
    }
}

// Block-jackknife standard errors of Re C and Im C at every lag.
__global__ void k_corr_cse(const double* C, int64_t n_lags, int B, double* cse) {
    const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= n_lags) return;
    for (int part = 0; part < 2; ++part) {
        double se = NAN;
        if (B >= 2) {
            double mean = 0.0;
            for (int b = 1; b <= B; ++b) mean += C[2 * ((int64_t)b * n_lags + l) + part];
            mean /= B;
            double v = 0.0;
            for (int b = 1; b <= B; ++b) {
                const double d = C[2 * ((int64_t)b * n_lags + l) + part] - mean;
                v += d * d;
            }
            se = sqrt((double)(B - 1) / B * v);
        }
        cse[2 * l + part] = se;
    }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Trajectory rows of a context: x and y rows of trajectory m start at
// x + m xs and y + m xs; z rows at z + m N.
struct Rows {
    void *x, *y, *z;
    int64_t xs;
};

Rows rows_of(twa_ctx* c) {
    if (c->tc) return Rows{c->tc->X, c->tc->Y, c->tc->Z, c->N};
    return Rows{c->xy, c->xy + c->N, c->z, 2 * c->N};
}

// Copy the state of A into B and C with the kicks, and give B and C A's step.
int kick_copies(twa_ctx* A, twa_ctx* B, twa_ctx* C, double eps) {
    const Rows a = rows_of(A), b = rows_of(B), c = rows_of(C);
    const double c2 = cos(2.0 * eps), s2 = sin(2.0 * eps);
    const int64_t M = A->M, N = A->N;
    if (A->tc) {
        k_kick<float><<<nblk(M * N, 256), 256, 0, A->stream>>>(
            (const float*)a.x, (const float*)a.y, (const float*)a.z, a.xs, (float*)b.x, (float*)b.y, (float*)b.z,
            (float*)c.x, (float*)c.y, (float*)c.z, M, N, c2, s2);
    } else {
        k_kick<double><<<nblk(M * N, 256), 256, 0, A->stream>>>(
            (const double*)a.x, (const double*)a.y, (const double*)a.z, a.xs, (double*)b.x, (double*)b.y,
            (double*)b.z, (double*)c.x, (double*)c.y, (double*)c.z, M, N, c2, s2);
    }
    TWA_CUDA(A, cudaGetLastError());
    for (twa_ctx* k : {B, C}) {
        TWA_CUDA(A, cudaMemcpyAsync(k->d_t, A->d_t, sizeof(int64_t), cudaMemcpyDeviceToDevice, A->stream));
        k->steps = A->steps;
        const int rc = k->tc ? tc_state_changed(k) : f64_state_changed(k);
        if (rc) return set_error(A, rc, k->err);
    }
    return TWA_OK;
}

int corr_samples(twa_ctx* A, twa_ctx* B, twa_ctx* C, const double* s0, double* s0w, double inv_eps, double* q) {
    const Rows a = rows_of(A), b = rows_of(B), c = rows_of(C);
    const CorrRows r{a.x, a.y, b.x, b.y, c.x, c.y, a.xs};
    if (A->tc) k_corr_samples<float><<<nblk(32 * A->M, 256), 256, 0, A->stream>>>(r, A->M, A->N, s0, s0w, inv_eps, q);
    else k_corr_samples<double><<<nblk(32 * A->M, 256), 256, 0, A->stream>>>(r, A->M, A->N, s0, s0w, inv_eps, q);
    TWA_CUDA(A, cudaGetLastError());
    return TWA_OK;
}

}  // namespace
}  // namespace twa

extern "C" int twa_correlation(twa_ctx* ctx, const twa_corr_req* req, twa_corr_out* out, double* C, double* S,
                               double* parts, double* C_se) {
    using namespace twa;
    NvtxRange range("twa_correlation: three copies, lags, spectrum");
    if (!ctx || !req || !out) return set_error(ctx, TWA_EINVAL, "twa_correlation: NULL argument");
    const int64_t M = req->M;
    if (M < 1 || M > (int64_t)1 << 30) return set_error(ctx, TWA_EINVAL, "twa_correlation: M must be in [1, 2^30]");
    if (req->prep_steps < 0 || req->lag_steps < 0 || req->lag_stride < 1 ||
        req->prep_steps + req->lag_steps > 0xFFFFFFFFll)
        return set_error(ctx, TWA_EINVAL, "twa_correlation: bad step counts");
    if (!(req->eps > 0.0) || !(req->eps < 1.0))
        return set_error(ctx, TWA_EINVAL, "twa_correlation: eps must be in (0, 1)");
    if (req->n_omega < 3 || req->n_omega > (int64_t)1 << 24 || !(req->omega_max > 0.0) || isinf(req->omega_max))
        return set_error(ctx, TWA_EINVAL, "twa_correlation: need n_omega in [3, 2^24] and finite omega_max > 0");
    if (ctx->opts.traj_offset + M - 1 > 0xFFFFFFFFll)
        return set_error(ctx, TWA_EINVAL, "twa_correlation: traj_offset + M exceeds the 32-bit trajectory counter");
    const int64_t n_lags = 1 + req->lag_steps / req->lag_stride;
    const int B = (int)(M < CORR_JB ? M : CORR_JB);
    const int nest = B + 1;
    memset(out, 0, sizeof(*out));

    // the three copies: same parameters, seed, trajectory offset and options
    twa_ctx* cp[3] = {nullptr, nullptr, nullptr};
    auto destroy = [&]() {
        for (twa_ctx*& k : cp) {
            twa_destroy(k);
            k = nullptr;
        }
    };
    twa_opts o = ctx->opts;
    o.window_start = 0.0;
    for (twa_ctx*& k : cp) {
        const int rc = twa_init(&k, ctx->N, ctx->alpha, ctx->w, ctx->Gamma, ctx->dt, ctx->seed, &o);
        if (rc) {
            set_error(ctx, rc, std::string("twa_correlation: ") + twa_last_error(nullptr));
            destroy();
            return rc;
        }
    }
    twa_ctx *A = cp[0], *Bc = cp[1], *Cc = cp[2];
    cudaStream_t st = ctx->stream;
    int rc = TWA_OK;
    {
        Scratch<double> s0(ctx, st), q(ctx, st), acc(ctx, st), pm(ctx, st), cc(ctx, st), sp(ctx, st), wd(ctx, st),
            cse(ctx, st);
        auto fail = [&](int code, const std::string& msg) {
            set_error(ctx, code, "twa_correlation: " + msg);
            return code;
        };
        auto run = [&](twa_ctx* k, int64_t steps) {
            const int r = twa_run(k, M, steps);
            if (r) set_error(ctx, r, "twa_correlation: " + k->err);
            return r;
        };
        if (s0.alloc(sizeof(double) * 2 * M) || q.alloc(sizeof(double) * CORR_Q * M) ||
            acc.alloc(sizeof(double) * CORR_Q * B * n_lags) || pm.alloc(sizeof(double) * CORR_Q * nest * n_lags) ||
            cc.alloc(sizeof(double) * 2 * nest * n_lags) || sp.alloc(sizeof(double) * nest * req->n_omega) ||
            wd.alloc(sizeof(double) * 8) || cse.alloc(sizeof(double) * 2 * n_lags))
            rc = fail(TWA_ENOMEM, "device scratch");
        // preparation of A, then the copies at the kick
        if (!rc) rc = run(A, req->prep_steps);
        if (!rc) rc = run(Bc, 0);
        if (!rc) rc = run(Cc, 0);
        if (!rc && (rc = kick_copies(A, Bc, Cc, req->eps))) set_error(ctx, rc, "twa_correlation: " + A->err);
        if (!rc && (rc = corr_samples(A, Bc, Cc, nullptr, s0.p, 0.0, nullptr)))
            set_error(ctx, rc, "twa_correlation: " + A->err);
        const double inv_eps = 1.0 / req->eps;
        for (int64_t l = 0; l < n_lags && !rc; ++l) {
            if (l > 0) {
                for (twa_ctx* k : cp)
                    if ((rc = run(k, req->lag_stride))) break;
                if (rc) break;
            }
            if ((rc = corr_samples(A, Bc, Cc, s0.p, nullptr, inv_eps, q.p))) {
                set_error(ctx, rc, "twa_correlation: " + A->err);
                break;
            }
            k_corr_blocks<<<B, 256, 0, st>>>(q.p, M, B, acc.p + l * B * CORR_Q);
            if (cudaGetLastError() != cudaSuccess) rc = fail(TWA_ECUDA, "block sums");
        }
        if (!rc) {
            k_corr_means<<<nblk((int64_t)nest * n_lags, 256), 256, 0, st>>>(acc.p, n_lags, B, M, pm.p, cc.p);
            k_corr_spectrum<<<nblk((int64_t)nest * req->n_omega, 128), 128, 0, st>>>(
                cc.p, n_lags, nest, req->n_omega, req->omega_max, (double)req->lag_stride * ctx->dt, sp.p);
            k_corr_width<<<1, 64, 0, st>>>(sp.p, nest, req->n_omega, req->omega_max, wd.p);
            k_corr_cse<<<nblk(n_lags, 256), 256, 0, st>>>(cc.p, n_lags, B, cse.p);
            if (cudaGetLastError() != cudaSuccess) rc = fail(TWA_ECUDA, "spectrum kernels");
        }
        double res[4] = {0, 0, 0, 0};
        if (!rc) {
            cudaError_t e = cudaMemcpyAsync(res, wd.p, sizeof(res), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && C)
                e = cudaMemcpyAsync(C, cc.p, sizeof(double) * 2 * n_lags, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && S)
                e = cudaMemcpyAsync(S, sp.p, sizeof(double) * req->n_omega, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && parts)
                e = cudaMemcpyAsync(parts, pm.p, sizeof(double) * CORR_Q * n_lags, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && C_se)
                e = cudaMemcpyAsync(C_se, cse.p, sizeof(double) * 2 * n_lags, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_check(ctx, e, "twa_correlation: results");
        }
        // device-side errors of the three runs (non-finite spins, timeouts)
        for (twa_ctx* k : cp)
            if (!rc && (rc = twa_sync(k))) set_error(ctx, rc, "twa_correlation: " + k->err);
        if (!rc) {
            double c0[2] = {0, 0};
            if (cudaMemcpy(c0, cc.p, sizeof(c0), cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = fail(TWA_ECUDA, "results");
            out->n_lags = n_lags;
            out->dtau = (double)req->lag_stride * ctx->dt;
            out->fwhm = res[0];
            out->fwhm_se = res[1];
            out->omega_peak = res[2];
            out->S_peak = res[3];
            out->spsm_tau0 = c0[0];
            out->M = M;
        }
        cudaStreamSynchronize(st);   // the scratch below is released in stream order; the copies are freed next
    }
    destroy();
    return rc;
}

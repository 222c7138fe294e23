// Ensemble reduction of the per-trajectory window sums to the observables of
// Sec. S1 (items 5-6) and the main text: means over trajectories of the window
// means of S^z, <S+S-> = A + S^z/2, <S+S+S-S-> = A^2 + 2 A S^z - S^z/3 +
// (S^z)^2/2 - 4A/3; g2 = <S+S+S-S-> / <S+S->^2 as a ratio of ensemble means.
// Standard errors: sample standard deviation / sqrt(M) for the linear
// observables, delete-one block jackknife over min(32, M) contiguous blocks
// (block b = trajectories [b M / B, (b+1) M / B)) for g2. All FP64.
#include <math.h>
#include <string.h>

#include <string>

#include "twa_internal.cuh"

// Scratch of twa_reduce_moments_noalloc: [0] sample count (int64 bits),
// [8, 16) results, [16, 16 + 5 M) the per-trajectory window means. Held by every
// device that loads the library; shared by all calls on that device.
static __device__ __align__(256) double twa_noalloc_scratch[16 + 5 * (int64_t)TWA_NOALLOC_MAX_M];

namespace twa {
namespace {

constexpr int RT = 1024;
constexpr int JB = 32;

__device__ __forceinline__ void derived(const double* mu, double& spsm, double& g2n) {
    // mu = (S^z, A, A^2, A S^z, (S^z)^2)
    spsm = mu[1] + 0.5 * mu[0];
    g2n = mu[2] + 2.0 * mu[3] - mu[0] / 3.0 + 0.5 * mu[4] - 4.0 / 3.0 * mu[1];
}

__device__ double block_sum(double v, double* sm) {
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int k = RT / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
        __syncthreads();
    }
    const double r = sm[0];
    __syncthreads();
    return r;
}

// out: Sz, Sz_se, SpSm, SpSm_se, G2num, G2num_se, g2, g2_se
__global__ void __launch_bounds__(RT) k_observables(const double* mom, const int64_t* d_count, int64_t M,
                                                    double* out) {
    __shared__ double sm[RT];
    __shared__ double bsum[JB][5];
    const double inv = 1.0 / (double)(*d_count);
    // first pass: sums of the three linear per-trajectory samples and of the raw moments
    double s_sz = 0, s_sp = 0, s_g = 0;
    double raw[5] = {0, 0, 0, 0, 0};
    for (int64_t m = threadIdx.x; m < M; m += RT) {
        double mu[5];
        for (int k = 0; k < 5; ++k) mu[k] = mom[5 * m + k] * inv;
        double sp, g;
        derived(mu, sp, g);
        s_sz += mu[0];
        s_sp += sp;
        s_g += g;
    }
    const double mean_sz = block_sum(s_sz, sm) / M;
    const double mean_sp = block_sum(s_sp, sm) / M;
    const double mean_g = block_sum(s_g, sm) / M;
    // second pass: squared deviations
    double d_sz = 0, d_sp = 0, d_g = 0;
    for (int64_t m = threadIdx.x; m < M; m += RT) {
        double mu[5];
        for (int k = 0; k < 5; ++k) mu[k] = mom[5 * m + k] * inv;
        double sp, g;
        derived(mu, sp, g);
        d_sz += (mu[0] - mean_sz) * (mu[0] - mean_sz);
        d_sp += (sp - mean_sp) * (sp - mean_sp);
        d_g += (g - mean_g) * (g - mean_g);
    }
    const double v_sz = block_sum(d_sz, sm), v_sp = block_sum(d_sp, sm), v_g = block_sum(d_g, sm);
    // jackknife block sums of the raw window means, one warp per block
    const int B = (int)(M < JB ? M : JB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < B) {
        const int64_t lo = (int64_t)warp * M / B, hi = (int64_t)(warp + 1) * M / B;
        for (int k = 0; k < 5; ++k) raw[k] = 0;
        for (int64_t m = lo + lane; m < hi; m += 32)
            for (int k = 0; k < 5; ++k) raw[k] += mom[5 * m + k] * inv;
        for (int k = 0; k < 5; ++k)
            for (int o = 16; o; o >>= 1) raw[k] += __shfl_xor_sync(0xffffffffu, raw[k], o);
        if (lane == 0)
            for (int k = 0; k < 5; ++k) bsum[warp][k] = raw[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double rM = sqrt((double)M);
        out[0] = mean_sz;
        out[1] = (M > 1) ? sqrt(v_sz / (M - 1)) / rM : NAN;
        out[2] = mean_sp;
        out[3] = (M > 1) ? sqrt(v_sp / (M - 1)) / rM : NAN;
        out[4] = mean_g;
        out[5] = (M > 1) ? sqrt(v_g / (M - 1)) / rM : NAN;
        double tot[5] = {0, 0, 0, 0, 0};
        for (int b = 0; b < B; ++b)
            for (int k = 0; k < 5; ++k) tot[k] += bsum[b][k];
        double mu[5], sp, g;
        for (int k = 0; k < 5; ++k) mu[k] = tot[k] / M;
        derived(mu, sp, g);
        out[6] = g / (sp * sp);
        if (B >= 2) {
            double est[JB], ebar = 0;
            for (int b = 0; b < B; ++b) {
                const int64_t cnt = (int64_t)(b + 1) * M / B - (int64_t)b * M / B;
                for (int k = 0; k < 5; ++k) mu[k] = (tot[k] - bsum[b][k]) / (double)(M - cnt);
                derived(mu, sp, g);
                est[b] = g / (sp * sp);
                ebar += est[b];
            }
            ebar /= B;
            double v = 0;
            for (int b = 0; b < B; ++b) v += (est[b] - ebar) * (est[b] - ebar);
            out[7] = sqrt((double)(B - 1) / B * v);
        } else {
            out[7] = NAN;
        }
    }
}

}  // namespace

int reduce_observables(twa_ctx* c, twa_obs* o) {
    Scratch<double> d_buf(c, c->stream);
    TWA_CUDA(c, d_buf.alloc(8 * sizeof(double)));
    double* d = d_buf.p;
    k_observables<<<1, RT, 0, c->stream>>>(c->mom, c->d_count, c->M, d);
    TWA_CUDA(c, cudaGetLastError());
    double h[8];
    int64_t cnt = 0;
    TWA_CUDA(c, cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    TWA_CUDA(c, cudaMemcpyAsync(&cnt, c->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    TWA_CUDA(c, cudaStreamSynchronize(c->stream));
    o->Sz = h[0];
    o->Sz_se = h[1];
    o->sigma_z = h[0] / c->N;
    o->sigma_z_se = h[1] / c->N;
    o->SpSm = h[2];
    o->SpSm_se = h[3];
    o->G2num = h[4];
    o->G2num_se = h[5];
    o->g2 = h[6];
    o->g2_se = h[7];
    o->samples = cnt;
    return TWA_OK;
}

}  // namespace twa

namespace {
// Device address of the scratch array in the context current on this thread.
// The host-side symbol is only a stand-in, not a device address, and the device
// address belongs to one CUDA context: it changes after cudaDeviceReset and
// differs in a context the caller created itself. So it is looked up on every
// call; the lookup allocates nothing (the first lookup in a context loads the
// library's device code into that context).
int noalloc_base(double** base) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, twa_noalloc_scratch);
    if (e != cudaSuccess) return twa::cuda_check(nullptr, e, "twa_reduce_moments_noalloc: cudaGetSymbolAddress");
    *base = p;
    return TWA_OK;
}
}  // namespace

extern "C" int twa_reduce_moments_noalloc(const double* means, int64_t M, int64_t N, twa_obs* out) {
    if (!means || !out || M < 1 || N < 1)
        return twa::set_error(nullptr, TWA_EINVAL, "twa_reduce_moments_noalloc: NULL pointer, M < 1 or N < 1");
    if (M > TWA_NOALLOC_MAX_M)
        return twa::set_error(nullptr, TWA_EINVAL,
                              "twa_reduce_moments_noalloc: M = " + std::to_string((long long)M) +
                                  " exceeds the static scratch limit TWA_NOALLOC_MAX_M = " +
                                  std::to_string((long long)TWA_NOALLOC_MAX_M));
    double* base = nullptr;
    int rc = noalloc_base(&base);
    if (rc) return rc;
    const int64_t one = 1;
    cudaError_t e = cudaMemcpy(base, &one, sizeof(one), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + 16, means, sizeof(double) * 5 * M, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return twa::cuda_check(nullptr, e, "twa_reduce_moments_noalloc: upload");
    twa::k_observables<<<1, twa::RT>>>(base + 16, reinterpret_cast<const int64_t*>(base), M, base + 8);
    e = cudaGetLastError();
    if (e != cudaSuccess) return twa::cuda_check(nullptr, e, "twa_reduce_moments_noalloc: launch");
    double h[8];
    e = cudaMemcpy(h, base + 8, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return twa::cuda_check(nullptr, e, "twa_reduce_moments_noalloc: download");
    memset(out, 0, sizeof(*out));
    out->Sz = h[0];
    out->Sz_se = h[1];
    out->sigma_z = h[0] / N;
    out->sigma_z_se = h[1] / N;
    out->SpSm = h[2];
    out->SpSm_se = h[3];
    out->G2num = h[4];
    out->G2num_se = h[5];
    out->g2 = h[6];
    out->g2_se = h[7];
    out->M = M;
    out->samples = 1;
    return TWA_OK;
}

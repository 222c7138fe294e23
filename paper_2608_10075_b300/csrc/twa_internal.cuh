// Internal declarations of libtwa: the context, device helpers shared by the
// kernels, and the host launchers each .cu file provides.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "../../include/twa.h"

namespace twa {

// ---------------------------------------------------------------------------
// device flag words (ctx->d_flags)
enum : int {
    FLAG_NONFINITE = 0,   // spin components found NaN/Inf
    FLAG_TIMEOUT = 1,     // bounded waits that gave up
    FLAG_DONE = 2,        // last-block counter of the per-step closing kernel
    FLAG_NOTPSD = 3,      // Cholesky pivots <= 0 (count)
    FLAG_NOTPSD_IDX = 4,  // first failing pivot index + 1 (atomicMin-free: set once)
    FLAG_COUNT = 8
};

// Row tiles of the tensor-core path: 128 sites per tile.
constexpr int TC_BM = 128;
// Column tiles: 256 B-operand rows = 128 trajectories x (x, y).
constexpr int TC_BN = 256;
constexpr int TC_BK = 64;

// Buffers of the mixed-precision path (twa_tc.cu, twa_fft.cu).
struct TcState {
    int64_t M = 0, N = 0, ldk = 0, n_rt = 0;
    int terms = 3;                               // products per W entry: 1 (BF16, BF16L2, BF16B, TF32), 2 (BF16X2), 3 (BF16X3, FP32)
    int lterms = 2;                              // products per L entry: 1 (BF16, BF16B, TF32), 2, 3 (FP32)
    int band = 0;                                // BF16L2, BF16B: 64-column blocks on each side of a 256-row
                                                 // unit whose one-product entries take the lo product too
    int bn = 256, kc = 0;                        // tile width and K-stage configuration
    int pair = 0;                                // CTA pairs: 256-row tiles on clusters of two (cta_group::2)
    int num_sms = 148;
    int clusters = 0;                            // resident clusters of two of the pair kernel
    // images of W / w and L / sqrt(w) (w > 0; of W and L when w = 0): a change of
    // w leaves them bit for bit unchanged and enters only through the factors below
    __nv_bfloat16 *Whi = nullptr, *Wlo = nullptr, *Lhi = nullptr, *Llo = nullptr;   // [N][ldk]
    double wsc = 1.0, lsc = 1.0;   // W = wsc * (image of W), L = lsc * (image of L)
    float *X = nullptr, *Y = nullptr, *Z = nullptr;       // state [M][N]
    float *Xp = nullptr, *Yp = nullptr, *Zp = nullptr;    // predictor
    float *Bx = nullptr, *By = nullptr;                   // noise part of the field increment
    __nv_bfloat16 *Shi = nullptr, *Slo = nullptr;         // images of s   [2M][ldk]
    __nv_bfloat16 *Phi = nullptr, *Plo = nullptr;         // images of s~  [2M][ldk]
    // noise images: eta of step s in E (s even) or E1 (s odd) on the dense route,
    // so that the draw of step t + 2 can run while the launches of step t read
    // step t + 1's; the FFT route uses E alone
    __nv_bfloat16* E = nullptr;                           // eta           [2M][ldk]
    __nv_bfloat16* Elo = nullptr;                         // lo image of eta (FP32 mode only)
    float* XI = nullptr;                                  // [M][2] collective normals
    __nv_bfloat16 *E1 = nullptr, *Elo1 = nullptr;         // the odd-step buffers
    float* XI1 = nullptr;
    CUtensorMap tmE1, tmElo1;
    // the noise draw of step t + 2 on a second stream beside step t's launches
    // (TWA_NOISE_OVERLAP = 0: on the context's stream, before them)
    bool overlap_noise = true;
    bool noise_epi = true;                       // dense step: the noise of t + 2 drawn inside the MIX launches
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    float* part = nullptr;                                // [n_rt][M][4] sums of s
    float* partp = nullptr;                               // [n_rt][M][4] sums of s~
    CUtensorMap tmWhi, tmWlo, tmLhi, tmLlo, tmShi, tmSlo, tmPhi, tmPlo, tmE, tmElo;
    // extra N x N operands (the adjoint's dW/dalpha and dL/dalpha), hi/lo images
    __nv_bfloat16 *Xhi[2] = {nullptr, nullptr}, *Xlo[2] = {nullptr, nullptr};
    CUtensorMap tmXhi[2], tmXlo[2];
    // vector images for tc_contract_f32 (rows fixed at first use)
    int64_t vec_rows = 0;
    __nv_bfloat16 *Vhi = nullptr, *Vlo = nullptr;
    CUtensorMap tmVhi, tmVlo;
    // dense step: the L.eta tiles of step t + 1 share the predictor's and the
    // corrector's launches of step t, so the noise part alternates between two
    // buffers, (Bx, By) for even steps and (Bx1, By1) for odd ones
    float *Bx1 = nullptr, *By1 = nullptr;
    int64_t bn_ready = -1;          // step whose noise part is in its buffer (-1: none)
    bool separate_leta = false;     // run L.eta as a launch of its own each step instead
    struct MixPlan* mix = nullptr;  // descriptor tables and tile schedules of the two launches
};

// Circulant-embedding FFT plan of the Toeplitz pump matrix (twa_fft.cu).
struct FftPlan {
    int64_t P = 0;               // transform length: smallest 2^a 3^b 5^c >= max(2, 2N - 2), even (one CTA)
                                 // or a multiple of 4 C (a cluster of C CTAs per trajectory)
    int C = 1;                   // CTAs per trajectory: 1, or 2, 4, 8 for P > 28000 (thread-block cluster)
    unsigned local_mask = 0;     // bit s: the stage of stride P / (r_0 ... r_s) stays inside one CTA
    int wl = 0;                  // one CTA: stages s >= wl run warp by warp (nst: none)
    int64_t Lw = 0;              // block span of stage wl (each warp owns whole blocks)
    // one CTA: direct twiddle tables w_L^j, j < m_s, of the stages whose tables fit
    // the shared memory left beside the transform (dtw_off[s] = -1: two-level lookup)
    float2* dtw = nullptr;
    int dtw_off[40];
    int64_t dtw_total = 0;
    int nst = 0;                 // number of stages
    int radix[40] = {0};         // radix of each stage (DIF order)
    float* lam = nullptr;        // spectrum of the embedding, in the DIF output order
    float2* tw = nullptr;        // exp(-2 pi i n / P), n < P
    // circulant noise draw, in the same (digit-reversed) order as lam
    float* nscale = nullptr;     // sqrt(max(lam_k, 0) / P)
    int32_t* nfreq = nullptr;    // frequency k held at each position
};

}  // namespace twa

struct twa_ctx {
    // parameters (Eq. 2 and Eq. S1)
    int64_t N = 0;
    double alpha = 0, w = 0, Gamma = 0, dt = 0;
    uint64_t seed = 0;
    twa_opts opts{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;

    // set-up products (FP64, [N][N])
    double* W64 = nullptr;
    double* L64 = nullptr;
    double w_max = 0, w_min = 0, min_pivot = 0;
    int64_t clipped = 0;
    double factor_residual = 0;   // ||W - L L^T||_F / ||W||_F when columns were clipped, else 0

    // run state
    int64_t M = 0;           // 0 until the first run / set_state
    int64_t steps = 0;       // completed steps (host mirror of d_t)
    int64_t n_window = 0;    // samples after step t are taken when t > n_window ...
    int64_t n_stride = 1;    // ... and n_stride divides t - n_window
    int64_t* d_t = nullptr;  // device step counter
    unsigned long long* d_flags = nullptr;
    double* mom = nullptr;   // [M][5] window sums (FP64)
    int64_t* d_count = nullptr;  // window samples taken (device)

    // FP64 path buffers
    double* xy = nullptr;    // [2M][N]: row 2m = x of trajectory m, 2m+1 = y
    double* z = nullptr;     // [M][N]
    double* xyp = nullptr;   // predictor
    double* zp = nullptr;
    double* hxy = nullptr;   // s + f(s)/2
    double* hz = nullptr;
    double* eta = nullptr;   // [2M][N] normals, then L.eta, then the noise part of B
    double* pf = nullptr;    // [2M][N] pump field W.s
    double* xi = nullptr;    // [M][2] collective normals
    double* S = nullptr;     // [M][4] collective sums of the current state
    double* Sp = nullptr;    // [M][4] collective sums of the predictor

    // resident route: FP32 copies of W and L (NULL on the other routes), or the
    // tensor-core form (BF16X2, N <= TWA_RESIDENT_TC_MAX_N) on the images of tc
    float* res_W = nullptr;
    float* res_L = nullptr;
    bool res_tc = false;

    // tensor-core (BF16 / BF16X3) path, and the FFT plan of the Toeplitz route
    twa::TcState* tc = nullptr;
    twa::FftPlan* fft = nullptr;

    // one captured step, replayed by twa_run (no host launch overhead per kernel)
    cudaGraphExec_t step_graph[2] = {nullptr, nullptr};   // captured step, by parity of the step index
    cudaStream_t capture_stream = nullptr;
    bool graph_failed = false;

    // per-launch event timing (twa_profile)
    struct ProfRec {
        int kind;
        cudaEvent_t a, b;
        double flops;   // tensor-core FLOPs the launch issues (0: none)
        double alg;     // algorithmic FLOPs of its contractions (counted once)
    };
    bool profiling = false;
    std::vector<ProfRec> prof;
};

namespace twa {
// NVTX range over one phase of a call (set-up, factor, step block, reduction,
// reverse sweep), for timeline tools; costs nothing when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Brackets one launch with CUDA events on the context's stream when profiling.
struct ProfScope {
    twa_ctx* c;
    int kind;
    double flops, alg;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(twa_ctx* ctx, int k, double fl = 0.0, double al = 0.0) : c(ctx), kind(k), flops(fl), alg(al) {
        if (c->profiling && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, c->stream);
    }
    ~ProfScope() {
        if (c->profiling && a && b) {
            cudaEventRecord(b, c->stream);
            c->prof.push_back({kind, a, b, flops, alg});
        }
    }
};
}  // namespace twa

namespace twa {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): a 10-round bijection of a
// 128-bit counter under a 64-bit key. Round: (c0, c1, c2, c3) ->
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key is
// bumped by the Weyl constants between rounds.
__host__ __device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Pump/collective noise stream 0 and initial-sign stream 1 (see twa.h).
constexpr uint32_t STREAM_NOISE = 0;
constexpr uint32_t STREAM_INIT = 1;
constexpr uint32_t STREAM_CIRCULANT = 2;   // circulant noise draw: counter (m, t, frequency k, 2)

// The state after step t1 is a window sample (the averaging window of Sec. S1).
__host__ __device__ __forceinline__ bool window_sample(int64_t t1, int64_t n_window, int64_t stride) {
    return t1 > n_window && (t1 - n_window) % stride == 0;
}

// Two FP64 standard normals from one Philox call: 53-bit uniforms
// u = (k + 1/2) 2^-53 from words (0,1) and (2,3), then Box-Muller.
__device__ __forceinline__ void normal2_f64(uint64_t seed, uint32_t m, uint32_t t, uint32_t i,
                                            double& gx, double& gy) {
    const uint4 r = philox10(make_uint4(m, t, i, STREAM_NOISE), (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t k1 = ((((uint64_t)r.x) << 32) | r.y) >> 11;
    const uint64_t k2 = ((((uint64_t)r.z) << 32) | r.w) >> 11;
    const double u1 = ((double)k1 + 0.5) * 0x1p-53;
    const double u2 = ((double)k2 + 0.5) * 0x1p-53;
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    gx = rad * c;
    gy = rad * s;
}

// FP32 variant from the same Philox words (words 0 and 2 as 32-bit uniforms in
// (0, 1]); used by the mixed-precision path, whose noise is rounded to BF16.
__device__ __forceinline__ void normal2_f32(uint64_t seed, uint32_t m, uint32_t t, uint32_t i,
                                            float& gx, float& gy, uint32_t stream = STREAM_NOISE) {
    const uint4 r = philox10(make_uint4(m, t, i, stream), (uint32_t)seed, (uint32_t)(seed >> 32));
    const float u1 = fmaf((float)r.x, 0x1p-32f, 0x1p-33f);
    const float u2 = fmaf((float)r.z, 0x1p-32f, 0x1p-33f);
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    gx = rad * c;
    gy = rad * s;
}

// Midpoint m = (s + s')/2 of the implicit-midpoint rotation s' = s + m x b, b =
// (B^y, -B^x, 0) (Mentink et al. 2010): with c = b/2, m - m x c = s gives
// m = (s + s x c + (s.c) c) / (1 + |c|^2), s x c = (z B^x, z B^y, -(x B^x +
// y B^y)) / 2, s.c = (x B^y - y B^x) / 2. Every rounding written out, so that
// each kernel instantiation gives the same bits.
__device__ __forceinline__ void mid_rotation_f32(float x, float y, float z, float Bx, float By, float& mx, float& my,
                                                 float& mz) {
    const float hx = __fmul_rn(0.5f, Bx), hy = __fmul_rn(0.5f, By);
    const float sc = fmaf(x, hy, -__fmul_rn(y, hx));
    const float inv = __frcp_rn(fmaf(hx, hx, fmaf(hy, hy, 1.0f)));
    mx = __fmul_rn(fmaf(sc, hy, fmaf(z, hx, x)), inv);
    my = __fmul_rn(fmaf(-sc, hx, fmaf(z, hy, y)), inv);
    mz = __fmul_rn(fmaf(-x, hx, fmaf(-y, hy, z)), inv);
}

// Discrete-Wigner signs of site i of trajectory m: low bits of words 0 and 1.
__device__ __forceinline__ void init_signs(uint64_t seed, uint32_t m, uint32_t i, double& sx, double& sy) {
    const uint4 r = philox10(make_uint4(m, 0u, i, STREAM_INIT), (uint32_t)seed, (uint32_t)(seed >> 32));
    sx = (r.x & 1u) ? 1.0 : -1.0;
    sy = (r.y & 1u) ? 1.0 : -1.0;
}

// ---------------------------------------------------------------------------
// Device memory of a context: through the caller's allocator when twa_opts
// names one, else cudaMalloc / cudaFree for buffers that live with the context
// and cudaMallocAsync / cudaFreeAsync (ordered on `st`) for scratch of one call.
// A request of 0 bytes gives NULL and succeeds.
cudaError_t dev_malloc(twa_ctx* c, void** p, size_t bytes);
void dev_free(twa_ctx* c, void* p);
cudaError_t dev_malloc_async(twa_ctx* c, void** p, size_t bytes, cudaStream_t st);
void dev_free_async(twa_ctx* c, void* p, cudaStream_t st);
template <class T>
cudaError_t dev_malloc(twa_ctx* c, T** p, size_t bytes) {
    return dev_malloc(c, reinterpret_cast<void**>(p), bytes);
}
template <class T>
cudaError_t dev_malloc_async(twa_ctx* c, T** p, size_t bytes, cudaStream_t st) {
    return dev_malloc_async(c, reinterpret_cast<void**>(p), bytes, st);
}

// Scratch buffer of one call, released in stream order on `st` when the scope
// ends, on the error paths too.
template <class T>
struct Scratch {
    twa_ctx* c;
    cudaStream_t st;
    T* p = nullptr;
    Scratch(twa_ctx* ctx, cudaStream_t s) : c(ctx), st(s) {}
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    cudaError_t alloc(size_t bytes) { return dev_malloc_async(c, &p, bytes, st); }
    ~Scratch() { dev_free_async(c, p, st); }
};

// ---------------------------------------------------------------------------
// host launchers
// twa_setup.cu
int setup_pump(twa_ctx* c);                      // W64, L64, pivots, spectrum
// twa_fp64.cu
int f64_alloc(twa_ctx* c);
void f64_free(twa_ctx* c);
int f64_init_state(twa_ctx* c);
int f64_run(twa_ctx* c, int64_t steps);
int f64_state_changed(twa_ctx* c);               // recompute sums after set_state
// which: 0 = W (the pump field), 1 = L (the noise factor)
int f64_field(twa_ctx* c, const double* s, double* P, int64_t K, int which = 0);
void gemm_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
              int64_t n_i, int64_t n_n, int64_t K, double alpha, double beta, bool tri_a, bool lower_only,
              cudaStream_t st);
// twa_tc.cu
int tc_prepare(twa_ctx* c);                      // BF16 images of W and L
int tc_alloc(twa_ctx* c);
void tc_free_run(twa_ctx* c);                    // trajectory buffers only
void tc_free(twa_ctx* c);                        // everything, including the images
int tc_init_state(twa_ctx* c);
int tc_run(twa_ctx* c, int64_t t0, int64_t steps);   // steps t0 .. t0 + steps - 1, launched directly
// Graph support: tc_launch_step(c, t) launches step t with no host bookkeeping;
// on the dense route it needs tc_prime(c, t) first, and tc_steps_done(c, t + n)
// records after n steps that the noise part of step t + n is in its buffer.
int tc_prime(twa_ctx* c, int64_t t);
int tc_launch_step(twa_ctx* c, int64_t t);
void tc_steps_done(twa_ctx* c, int64_t t_next);
int tc_state_changed(twa_ctx* c);
int tc_get_state(twa_ctx* c, double* sx, double* sy, double* sz);   // device buffers
int tc_set_state(twa_ctx* c, const double* sx, const double* sy, const double* sz);
int tc_field(twa_ctx* c, const double* s, double* P, int64_t K, int which = 0);
// out[k] = A in[k] for FP32 device vectors [K][N] with BF16X3 (or BF16) tensor-core
// contractions; which: 0 = W, 1 = L (lower), 2, 3 = the extra matrices below.
int tc_contract_f32(twa_ctx* c, int which, const float* in, float* out, int64_t K);
int tc_set_extra_matrix(twa_ctx* c, int slot, const double* A64);   // slot 0 or 1, [N][N] FP64
// batches of contexts advanced by grouped launches (twa_tc.cu)
struct TcBatch;
int tc_batch_build(twa_ctx* const* ctxs, int n, twa_ctx* lead, TcBatch** out);
int tc_batch_prime(twa_ctx* lead, TcBatch* b, int64_t t);   // noise part of the batch's first step t
int tc_batch_step(twa_ctx* lead, TcBatch* b, int64_t t);    // step t of every context: 5 launches
void tc_batch_free(TcBatch* b);
int tc_set_tiles(twa_ctx* c, int bn, int kc);
int wait_probe(twa_ctx* c, int64_t limit_ns);    // one bounded wait that runs out (twa_wait_probe)
// twa_fft.cu
int fft_prepare(twa_ctx* c);                     // plan, twiddles, spectrum of the embedding
void fft_free(twa_ctx* c);
int fft_predict(twa_ctx* c);                     // W.s by FFT + Heun predictor (one step)
int fft_correct(twa_ctx* c);                     // W.s~ by FFT + corrector + moments (one step)
int fft_noise(twa_ctx* c);                       // circulant noise draw -> noise part (one step)
int fft_field(twa_ctx* c, const double* s, double* P, int64_t K);
// twa_resident.cu (resident route)
bool res_config(int64_t N, int* T, bool* resident, size_t* smem);
int res_prepare(twa_ctx* c);                     // FP32 copies of W and L
void res_free(twa_ctx* c);
int res_run(twa_ctx* c, int64_t steps);          // all steps in one launch
// steps[k] steps of each resident context cs[k] in one launch per CTA shape
int res_run_many(twa_ctx* const* cs, const int64_t* steps, int n, twa_ctx* lead, cudaStream_t st);
// twa_restc.cu (resident route on the tensor cores)
bool restc_capable(const twa_ctx* c);            // BF16X2 and N <= TWA_RESIDENT_TC_MAX_N
int restc_run_many(twa_ctx* const* cs, const int64_t* steps, int n, twa_ctx* lead, cudaStream_t st);
// twa_adjoint.cu
int grad(twa_ctx* c, const twa_grad_req* r, twa_grad_out* out, double* per_traj);
// twa_reduce.cu
int reduce_observables(twa_ctx* c, twa_obs* out);  // device FP64 reduction, synchronises

// error helpers (twa_api.cu)
int set_error(twa_ctx* c, int code, const std::string& msg);
int cuda_check(twa_ctx* c, cudaError_t e, const char* what);

}  // namespace twa

#define TWA_CUDA(c, call)                                              \
    do {                                                               \
        cudaError_t e__ = (call);                                      \
        if (e__ != cudaSuccess) return ::twa::cuda_check((c), e__, #call); \
    } while (0)

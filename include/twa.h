/*
 * twa.h - C ABI of libtwa, a single-GPU (sm_103a) engine for the dissipative
 * truncated-Wigner (TWA) dynamics of N spins under collective cavity decay and
 * a spatially correlated pump (arxiv 2608.10075).
 *
 * Model (Eq. 1, Eq. 2): collective decay at rate Gamma through S^- = sum_i
 * sigma_i^-, pump matrix w_ij = w / (|i-j| + 1)^alpha on an open chain.
 * Dynamics (Sec. S1, Eq. S1): every trajectory m carries classical spins
 * s_i = (x_i, y_i, z_i), i < N, moved by
 *     d x_i =  z_i B^x_i,   d y_i = z_i B^y_i,   d z_i = -(x_i B^x_i + y_i B^y_i),
 *     B^a_i  = 1/2 (Gamma S^a - sum_j w_ij s^a_j) dt + sqrt(Gamma dt) xi^a
 *              - sqrt(dt) (L eta^a)_i,           a = x, y,
 * with S^a = sum_j s^a_j, one collective normal xi^a per trajectory and step
 * (the noise <xi xi> = Gamma has no site index), eta^a iid normals per site,
 * and L L^T = W. Integrator: stochastic Heun (Stratonovich), then every spin is
 * rescaled to length sqrt(3). Initial state (Sec. S1, item 3): x, y = +-1,
 * z = init_state. Observables (Sec. S1, items 5-6, main text): window and
 * ensemble means of S^z, <S+S-> = A + S^z/2 and
 * <S+S+S-S-> = A^2 + 2 A S^z - S^z/3 + (S^z)^2/2 - 4/3 A, with A = |S^x + i S^y|^2/4,
 * and g2 = <S+S+S-S-> / <S+S->^2.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed low 32
 * bits, seed high 32 bits), counter = (trajectory m, step t, site i, stream).
 * Stream 0 gives the pump noise (i < N) and the collective noise (i = N),
 * stream 1 (t = 0) the initial signs. Results depend only on (parameters, seed,
 * m, t), never on launch shapes, so runs can be continued or split by
 * trajectory and reproduce one uninterrupted run.
 *
 * Conventions for every entry point:
 *  - Return 0 on success or a negative TWA_E* code; no exception crosses the
 *    ABI. After an error, twa_last_error(ctx) holds a one-line message. The
 *    context stays usable after TWA_EINVAL.
 *  - The library owns every device buffer it allocates (cudaMalloc on the
 *    current device at twa_init); twa_destroy frees them. Caller buffers are
 *    only read or written during the call that receives them (device buffers:
 *    in stream order on the context's stream).
 *  - Work is enqueued on the stream given in twa_opts (NULL = the legacy
 *    default stream). twa_run only enqueues; errors raised on the device
 *    (non-finite spins, a timed-out wait) are reported by the next call that
 *    synchronises: twa_sync, twa_observables, twa_get_state, twa_get_moments.
 *  - State arrays are [M][N] row-major: element (m, i) at m*N + i.
 */
#ifndef TWA_H
#define TWA_H

#include <stdint.h>

#if defined(__GNUC__)
#define TWA_API __attribute__((visibility("default")))
#else
#define TWA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define TWA_OK            0
#define TWA_EINVAL       -1  /* bad argument; nothing was changed            */
#define TWA_ENOTPSD      -2  /* the pump matrix has a non-positive pivot     */
#define TWA_ENOMEM       -3  /* device allocation failed                     */
#define TWA_ECUDA        -4  /* a CUDA call failed (message names it)        */
#define TWA_ETIMEOUT     -5  /* a device-side wait ran out of its time limit */
#define TWA_ENONFINITE   -6  /* a spin component became NaN or Inf           */
#define TWA_ESTATE       -7  /* call out of order (e.g. no trajectories yet) */
#define TWA_EUNSUPPORTED -8  /* option not available for these parameters   */

/* arithmetic of the per-step contractions W.S and L.eta */
#define TWA_PREC_FP64    0   /* FP64 everywhere (SIMT DFMA)                              */
#define TWA_PREC_BF16    1   /* tcgen05 BF16 x BF16 -> FP32, one term, FP32 state        */
#define TWA_PREC_BF16X3  2   /* tcgen05 split hi+lo: hi*hi + hi*lo + lo*hi, FP32 state   */
#define TWA_PREC_TF32    3   /* tcgen05 TF32 x TF32 -> FP32, one term, FP32 state; W, L,
                                s and eta rounded to TF32 (11 significant bits, relative
                                error 2^-11 against 2^-8 for BF16). Dense and FFT routes
                                of twa_init / twa_run / twa_field; not twa_grad,
                                twa_batch_run or the extra-matrix contractions        */
#define TWA_PREC_FP32    4   /* FP32-accurate contractions on tcgen05: every operand
                                (W, L, s, eta) split into TF32 hi = tf32(v) and lo =
                                tf32(v - hi), products hi*hi + hi*lo + lo*hi with FP32
                                accumulation (about 2^-22 relative per product, the
                                order of an FP32 product), FP32 state. Same coverage
                                as TWA_PREC_TF32                                      */
#define TWA_PREC_BF16X2  5   /* W and L held as BF16 hi + lo, their operand (the state,
                                the noise) rounded once to BF16: two products per entry,
                                A_hi*v + A_lo*v, FP32 accumulation, FP32 state. W.s is
                                W.bf16(s) to ~2^-17; L.eta is the BF16X3 arithmetic.
                                twa_run, twa_field, twa_contract, twa_batch_run,
                                twa_grad                                             */
#define TWA_PREC_BF16L2  6   /* W one BF16 product (W_hi*s_hi) except within 64 columns
                                of the diagonal, where it takes W_lo*s_hi too (the
                                band: all W entries with j in [u - 64, u + 320) for
                                the 256 rows i in [u, u + 256), u a multiple of 256);
                                L split as in BF16X2 (L_hi*eta + L_lo*eta). The
                                largest entries of the Toeplitz W, whose one-term
                                rounding errors repeat on every row and bias the
                                steady state, keep ~16 bits. Same coverage as
                                TWA_PREC_BF16X2                                       */
#define TWA_PREC_BF16B   7   /* W and L each one BF16 product (A_hi*v) off the band of
                                TWA_PREC_BF16L2 and two (A_hi*v + A_lo*v) on it, their
                                operand rounded once to BF16, FP32 accumulation, FP32
                                state: ~1.03 products per entry of W and of L. Same
                                coverage as TWA_PREC_BF16X2                           */

typedef struct twa_ctx twa_ctx;   /* opaque, owned by the library */

/* Caller-supplied device allocator (e.g. a framework's caching allocator), so
   that a context's device memory comes from the caller's pool. alloc returns
   `bytes` of device memory usable in work ordered on `stream` (a cudaStream_t;
   NULL = legacy default stream), or NULL on failure; free releases a pointer
   that alloc returned, for reuse after the work already ordered on `stream`.
   `user` is the twa_opts.alloc_user pointer. The memory must be aligned to
   256 bytes as cudaMalloc's is (the tensor maps of the tensor-core path need
   16). Both are called from the thread that calls into the library (for
   twa_batch_run: from its set-up threads too, so they must be thread-safe). */
typedef void* (*twa_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*twa_free_fn)(void* ptr, void* stream, void* user);

typedef struct twa_opts {
    int    precision;       /* TWA_PREC_*; default TWA_PREC_FP64                      */
    int    init_state;      /* initial s^z: -1 ground (default) or +1 excited         */
    double window_start;    /* t0: the state after step t is averaged when
                               t > round(t0 / dt) (and the stride below divides
                               t - round(t0 / dt)); default 0                         */
    int    renormalize;     /* 1 (default): rescale every spin to sqrt(3) each step   */
    int    clip_negative;   /* 0 (default): non-positive Cholesky pivot -> TWA_ENOTPSD;
                               1: zero that column of L and carry on. This zeroes
                               pivots during the factorisation; it does not clip
                               eigenvalues of W. twa_obs reports the count
                               (clipped) and ||W - L L^T||_F / ||W||_F            */
    void*  stream;          /* cudaStream_t for all work; NULL = default stream       */
    int64_t traj_offset;    /* global index of trajectory 0 in the Philox counter
                               (default 0): shards of one ensemble use disjoint
                               offsets and reproduce the unsharded run exactly     */
    int    ws_route;        /* pump field sum_j w_ij s_j: TWA_ROUTE_DENSE (default,
                               any W) or TWA_ROUTE_FFT (uses that Eq. 2 is Toeplitz;
                               tensor-core precisions only; one CTA per trajectory
                               while 2N - 2 <= 28000, else a thread-block cluster
                               of 2, 4 or 8 CTAs holding the transform in their
                               shared memories; TWA_FFT_CLUSTER = 1, 2, 4 or 8 in
                               the environment forces the cluster size)            */
    int    noise_route;     /* draw of the pump noise chi (covariance w_ij dt, Sec. S1):
                               TWA_NOISE_CHOLESKY (default: chi = L eta) or
                               TWA_NOISE_CIRCULANT (FFT of the circulant embedding;
                               needs ws_route = TWA_ROUTE_FFT). The two draws have the
                               same law and different per-trajectory values.       */
    int64_t sample_stride;  /* window samples every sample_stride-th step: the states
                               after steps n_w + k, n_w + 2k, ... with n_w =
                               round(t0 / dt); 0 or 1 (default): every step        */
    twa_alloc_fn alloc;     /* NULL (default): the library allocates with cudaMalloc
                               (buffers that live with the context) and
                               cudaMallocAsync (scratch of one call). Non-NULL,
                               with `free`: every device allocation of the context
                               and of the calls made on it goes through alloc/free
                               instead (the context-less twa_reduce_moments keeps
                               the library's allocator)                           */
    twa_free_fn free;
    void*  alloc_user;      /* passed through to alloc and free                   */
    int    integrator;      /* TWA_INT_HEUN (default) or TWA_INT_MIDPOINT          */
} twa_opts;

/* Integrators of Eq. S1, written with its effective field: ds_i = s_i x b_i,
   b_i = (B^y_i, -B^x_i, 0) over one step, B^a_i = 1/2 (Gamma S^a - sum_j w_ij
   s^a_j) dt + sqrt(Gamma dt) xi^a - sqrt(dt) (L eta^a)_i, the same noise in
   both stages of a step.
   HEUN: s~ = s + s x b(s), s' = s + (s x b(s) + s~ x b(s~)) / 2 (stochastic
   Heun, Stratonovich), then |s_i| = sqrt(3) if renormalize is set.
   MIDPOINT: the semi-implicit scheme the paper uses (Mentink et al., J. Phys.:
   Condens. Matter 22, 176001 (2010)): s~ solves s~ = s + ((s + s~)/2) x b(s),
   s' solves s' = s + ((s + s')/2) x b((s + s~)/2); each stage is an exact
   rotation, m = (s + s x c + (s.c) c) / (1 + |c|^2) with c = b/2 and s' = 2m - s,
   so |s_i| is kept without renormalisation (renormalize still removes the
   rounding drift). The corrector field is that of the midpoint state, whose
   images the predictor hands to the second contraction (on the FFT route, the
   midpoint state is the second transform's input). twa_run on both routes and
   twa_batch_run; not twa_grad.                                                */
#define TWA_INT_HEUN     0
#define TWA_INT_MIDPOINT 1

#define TWA_ROUTE_DENSE 0   /* tensor-core contraction with the dense W          */
#define TWA_ROUTE_FFT   1   /* circulant-embedding FFT convolution, FP32 (any N
                                up to the library's limit of 60000)            */
#define TWA_ROUTE_RESIDENT 2 /* small systems (N <= TWA_RESIDENT_MAX_N), precision
                                TWA_PREC_FP32: every twa_run call is one launch in
                                which each CTA integrates its trajectories for all
                                steps with the state in shared memory (W and L too
                                when they fit, else streamed through it from L2);
                                W.s and L.eta as FP32 FMA chains, FP32 normals (not
                                rounded to BF16), FP32 state, FP64 moments. Heun
                                and midpoint; Cholesky noise draw. twa_field and
                                twa_contract on such a context run the FP32
                                tensor-core split. With precision TWA_PREC_BF16X2
                                and N <= TWA_RESIDENT_TC_MAX_N the same route runs
                                on the tensor cores: each CTA holds the BF16 hi + lo
                                images of W and L and the BF16 images of its 32
                                trajectories' state, predictor and noise in shared
                                memory, the two FP32 accumulators in TMEM and the
                                FP32 state in registers for all steps; the BF16X2
                                arithmetic of the dense route                       */
#define TWA_RESIDENT_MAX_N 512
#define TWA_RESIDENT_TC_MAX_N 128

/* Pump-noise draws. Circulant: on a circle of even length P >= 2N - 2 (the
   smallest 2^a 3^b 5^c), c_d = w / (1 + min(d, P - d))^alpha is the first row
   of a circulant whose leading N x N block is W and whose eigenvalues lam_k
   are >= 0 (the sequence is convex and decreasing on 0..P/2: Dietrich-Newsam).
   With (a_k, b_k) the Box-Muller pair of Philox counter (m, t, k, stream 2),
   Y_j = sum_k sqrt(lam_k / P) (a_k + i b_k) exp(+2 pi i j k / P), and
   chi^x_j = Re Y_j, chi^y_j = Im Y_j for j < N: one FP32 transform per
   trajectory and step instead of the L.eta contraction.                    */
#define TWA_NOISE_CHOLESKY  0
#define TWA_NOISE_CIRCULANT 1

/* kernel classes timed by twa_profile_read. On the dense mixed-precision
   route the predictor and corrector launches of step t also carry the L.eta
   tiles of step t + 1; TWA_PROF_NOISE_FACTOR then counts only the standalone
   L.eta launch that opens a run (and every step of the FFT route).           */
#define TWA_PROF_NOISE     0   /* Philox normals of a step                      */
#define TWA_PROF_PREDICT   1   /* W.s contraction + Heun predictor              */
#define TWA_PROF_CORRECT   2   /* W.s~ contraction + Heun corrector             */
#define TWA_PROF_CLOSE     3   /* collective sums + window moments              */
#define TWA_PROF_GEMM64    4   /* FP64 path: one SIMT contraction               */
#define TWA_PROF_ELEM64    5   /* FP64 path: elementwise / reduction kernels    */
#define TWA_PROF_NOISE_FACTOR 6 /* mixed path: L.eta contraction -> noise part  */
#define TWA_PROF_RESIDENT  7   /* resident route: one launch of all steps        */
#define TWA_PROF_KINDS     8

typedef struct twa_obs {
    /* ensemble means over trajectories of the per-trajectory window means, and
       their standard errors (g2: block jackknife over min(32, M) blocks)       */
    double Sz, Sz_se;           /* <S^z>                                        */
    double sigma_z, sigma_z_se; /* <S^z> / N                                    */
    double SpSm, SpSm_se;       /* <S+S->, normal ordered                       */
    double G2num, G2num_se;     /* <S+S+S-S->, normal ordered                   */
    double g2, g2_se;           /* <S+S+S-S-> / <S+S->^2                        */
    int64_t M;                  /* trajectories                                 */
    int64_t steps;              /* completed steps                              */
    int64_t samples;            /* steps inside the averaging window            */
    /* diagnostics of the pump matrix (Eq. 3 and below) and of the run          */
    double w_max, w_min;        /* extreme eigenvalues of w_ij (Lanczos)        */
    double w_tilde;             /* w_max / (Gamma N)                             */
    double stability;           /* max(Gamma N, w_max) dt (the paper asks < 0.05) */
    double min_pivot;           /* smallest Cholesky pivot L_ii^2               */
    int64_t clipped;            /* columns of L zeroed by clip_negative         */
    int64_t nonfinite;          /* spin components found non-finite             */
    double factor_residual;     /* ||W - L L^T||_F / ||W||_F when clip_negative
                                   zeroed columns (else 0, not computed)        */
    int64_t fft_length;         /* FFT route: circle length P of the embedding
                                   (the smallest 2^a 3^b 5^c >= 2N - 2 that is even
                                   when one CTA holds the transform, i.e. P <= 28000,
                                   else a multiple of 4 fft_ctas); 0 otherwise  */
    int64_t fft_ctas;           /* FFT route: CTAs per trajectory (1; 2, 4 or 8
                                   as a thread-block cluster); 0 otherwise      */
} twa_obs;

/* Fill *opts with the defaults listed above. Returns TWA_EINVAL if opts is NULL. */
TWA_API int twa_opts_default(twa_opts* opts);

/* Create a context for N sites (Eq. 2 pump with exponent alpha >= 0 or +INF,
 * prefactor w >= 0), collective decay Gamma >= 0, step dt > 0, Philox seed.
 * Builds W in FP64 on the device and factors it (L L^T = W, lower triangular;
 * alpha = 0: the exact rank-one factor L[:,0] = sqrt(w); alpha = +INF: sqrt(w) I),
 * and computes the spectrum diagnostics. For the BF16 modes it also stores the
 * BF16 hi/lo images of W / w and L / sqrt(w) (of W and L when w = 0; the
 * step multiplies by w and sqrt(w) in FP32, so contexts that differ only in w
 * hold the same images). On success *out owns all device memory.
 * Errors: TWA_EINVAL (bad numbers, N < 1, NULL out), TWA_ENOTPSD (a pivot
 * <= 0 without clip_negative), TWA_ENOMEM, TWA_ECUDA. */
TWA_API int twa_init(twa_ctx** out, int64_t N, double alpha, double w, double Gamma,
             double dt, uint64_t seed, const twa_opts* opts);

/* Advance trajectories 0..M-1 by `steps` stochastic-Heun steps of Eq. S1.
 * The first call fixes M (>= 1) and samples the discrete-Wigner initial state;
 * later calls must pass the same M and continue the same noise stream (the
 * step counter persists). Enqueue only. Errors: TWA_EINVAL (M changed, M < 1,
 * steps < 0), TWA_ENOMEM, TWA_ECUDA. */
TWA_API int twa_run(twa_ctx* ctx, int64_t M, int64_t steps);

/* Wait for the context's stream and report device-side errors:
 * TWA_ENONFINITE, TWA_ETIMEOUT, TWA_ECUDA. */
TWA_API int twa_sync(twa_ctx* ctx);

/* Reduce the per-trajectory window sums to the observables above (FP64 on the
 * device) and copy them into the caller's host struct *out. Synchronises.
 * Errors: TWA_ESTATE (no trajectories or no window sample yet), plus those of
 * twa_sync. */
TWA_API int twa_observables(twa_ctx* ctx, twa_obs* out);

/* Copy the current spins into caller buffers of M*N doubles each, layout
 * [M][N]; `on_device` = 1 for device pointers, 0 for host pointers.
 * Synchronises. Errors: TWA_ESTATE (no trajectories yet), TWA_EINVAL. */
TWA_API int twa_get_state(twa_ctx* ctx, double* sx, double* sy, double* sz, int on_device);

/* Replace the spins of all M trajectories (fixing M if no run happened yet)
 * from caller buffers of M*N doubles each, layout [M][N]. Values are used as
 * given (no renormalisation); the step counter and window sums are kept.
 * Errors: TWA_EINVAL (NULL pointer, M < 1 or M differs from the fixed M). */
TWA_API int twa_set_state(twa_ctx* ctx, int64_t M, const double* sx, const double* sy,
                  const double* sz, int on_device);

/* The same two calls for FP32 buffers of M*N floats each, layout [M][N]: the
 * state of the tensor-core precisions is FP32, so these copy it as it is (no
 * conversion; half the bytes of the FP64 calls). twa_get_state_f32
 * synchronises; twa_set_state_f32 synchronises for host buffers. Errors: as
 * the FP64 calls, and TWA_EUNSUPPORTED on a TWA_PREC_FP64 context (FP64 spins). */
TWA_API int twa_get_state_f32(twa_ctx* ctx, float* sx, float* sy, float* sz, int on_device);
TWA_API int twa_set_state_f32(twa_ctx* ctx, int64_t M, const float* sx, const float* sy,
                      const float* sz, int on_device);

/* Copy the per-trajectory window means, M*5 doubles [M][5] in the order
 * S^z, A, A^2, A S^z, (S^z)^2 (symmetric-ordered classical moments, Sec. S1
 * item 5), to a host (on_device = 0) or device buffer. Synchronises.
 * Errors: TWA_ESTATE (no trajectories or no window sample yet). */
TWA_API int twa_get_moments(twa_ctx* ctx, double* out, int on_device);

/* Pump-field contraction of Eq. S1, P[k][i] = sum_j w_ij s[k][j], for K
 * caller vectors s (device, [K][N] doubles) into P (device, [K][N] doubles),
 * computed with the context's precision path (FP64; the BF16 images of W
 * and an hi/lo split of s, or their TF32 images or TF32 hi/lo splits, with
 * FP32 accumulation). Enqueued on the context's
 * stream. Errors: TWA_EINVAL (NULL, K < 1). */
TWA_API int twa_field(twa_ctx* ctx, const double* s, double* P, int64_t K);

/* matrices of twa_contract */
#define TWA_MAT_W 0         /* the pump matrix w_ij of Eq. 2                     */
#define TWA_MAT_L 1         /* its noise factor L (L L^T = W, lower triangular)  */

/* The contractions of one step alone, P[k][i] = sum_j A_ij s[k][j] for K caller
 * vectors (device, [K][N] doubles) into P (device, [K][N] doubles), with A the
 * pump matrix (TWA_MAT_W: the pump field sum_j w_ij s_j of Eq. S1, the same
 * result as twa_field) or the noise factor (TWA_MAT_L: the correlated noise
 * chi = L eta of Sec. S1 before its sqrt(dt) scaling), in the arithmetic the
 * context's step uses for it:
 *  - FP64: DFMA (the K range of L stops at the diagonal);
 *  - BF16X3: W hi/lo against an hi/lo split of s (three products), or L hi/lo
 *    against s rounded once to BF16 (two products), FP32 accumulation;
 *  - BF16X2: W or L hi/lo against s rounded once to BF16 (two products);
 *  - BF16L2: W one BF16 product, two within 64 columns of the diagonal; L as
 *    in BF16X2;
 *  - BF16B: W and L one BF16 product, two within 64 columns of the diagonal;
 *  - BF16: one product of BF16 images; TF32: one product of TF32 images;
 *  - FP32: TF32 hi/lo splits of both operands (three products).
 * On the FFT route TWA_MAT_W runs the FFT convolution, TWA_MAT_L the dense
 * tensor-core contraction. Enqueued on the context's stream.
 * Errors: TWA_EINVAL (NULL, unknown matrix, K < 1). */
TWA_API int twa_contract(twa_ctx* ctx, int matrix, const double* s, double* P, int64_t K);

/* objectives of twa_grad */
#define TWA_OBJ_SPSM 0      /* <S+S->, window and ensemble mean, normal ordered */
#define TWA_OBJ_G2   1      /* g2 = <S+S+S-S-> / <S+S->^2                      */

typedef struct twa_grad_req {
    int     objective;      /* TWA_OBJ_SPSM or TWA_OBJ_G2                          */
    int     want_alpha;     /* 1: also dJ/dalpha (needs 0 < alpha < inf)           */
    int64_t M;              /* trajectories (Philox indices traj_offset + 0..M-1)  */
    int64_t steps;          /* steps from the discrete-Wigner start                */
    int64_t checkpoint;     /* steps between stored states; <= 0 selects 64       */
} twa_grad_req;

typedef struct twa_grad_out {
    double J;                       /* objective of the forward run                */
    double dJ_dw, dJ_dw_se;         /* pathwise derivative and standard error      */
    double dJ_dalpha, dJ_dalpha_se; /* (0 when want_alpha = 0)                     */
    int64_t M, steps, samples;      /* samples: steps inside the averaging window  */
    double mu[5];                   /* forward ensemble means of the window moments
                                       S^z, A, A^2, A S^z, (S^z)^2                 */
} twa_grad_out;

/* Pathwise gradient of a steady-state objective with respect to the pump
 * prefactor w and exponent alpha of Eq. 2 at fixed noise (an extension: the
 * paper computes no derivatives).
 *
 * Runs its own forward pass of `steps` stochastic-Heun steps from the initial
 * state (the same trajectories twa_run would produce: same seed, counters and
 * precision; it neither reads nor changes the state of twa_run), storing the
 * state every `checkpoint` steps, then the reverse sweep: each block is
 * recomputed from its checkpoint and the cotangent is pulled back through the
 * renormalisation, the Heun corrector and the predictor, with W.beta
 * contractions on the precision path of the context (FP64 SIMT, or the BF16,
 * BF16X3, BF16X2, BF16L2 or BF16B tensor-core arithmetic of the forward step with an
 * FP32 tape). Parameter derivatives use dW/dw = W/w,
 * dL/dw = L/(2w), dW/dalpha = -ln(1+|i-j|) W and the Cholesky derivative
 * dL = L Phi(L^-1 dW L^-T). The objective is linearised at the forward run's
 * ensemble means (g2 through the quotient rule).
 *
 * per_traj: NULL or a host array [M][2] receiving M times each trajectory's
 * contribution to (dJ/dw, dJ/dalpha); their mean is the returned derivative and
 * their standard deviation / sqrt(M) the returned SE. Synchronises.
 * Errors: TWA_EINVAL (NULL, M < 1, steps < 1), TWA_ESTATE (no step inside the
 * window), TWA_EUNSUPPORTED (want_alpha with alpha = 0 or inf, w = 0, a
 * context with noise_route = TWA_NOISE_CIRCULANT, precision = TWA_PREC_TF32
 * or TWA_PREC_FP32, or integrator = TWA_INT_MIDPOINT),
 * TWA_ENOMEM, TWA_ECUDA,
 * TWA_ENONFINITE. */
TWA_API int twa_grad(twa_ctx* ctx, const twa_grad_req* req, twa_grad_out* out, double* per_traj);

/* one point of a batched scan */
typedef struct twa_point {
    int64_t N;              /* sites                                               */
    double  alpha, w;       /* pump matrix of Eq. 2                                */
    double  Gamma, dt;      /* collective decay, time step                         */
    int64_t steps;          /* steps to run from the discrete-Wigner start          */
    double  window_start;   /* averaging window start time (as twa_opts)           */
    double* means;          /* NULL, or a host array [M][5] that receives the point's
                               per-trajectory window means (twa_get_moments order) */
} twa_point;

/* Run many parameter points of uneven N together (e.g. a phase-diagram scan) and return each point's observables in out[0..n-1].
 *
 * Every point gets its own pump matrix, Cholesky factor and M trajectories (set
 * up concurrently from several host threads, each on its own stream; seed
 * and opts as for twa_init; opts->precision must be TWA_PREC_BF16,
 * TWA_PREC_BF16X3, TWA_PREC_BF16X2, TWA_PREC_BF16L2 or TWA_PREC_BF16B, opts->window_start is replaced by each point's, and every
 * point runs the dense route with the Cholesky noise draw). A step of all
 * points still running is the single-context step done for all of them at
 * once: noise of the next step, one persistent launch with every point's W.s +
 * predictor tiles and part of the L.eta tiles of the next step, one with the
 * W.s~ + corrector tiles and the rest (tiles placed on one CTA per SM by
 * longest-first list scheduling), window moments. The step is captured per
 * set of running points and parity of the step index as CUDA graphs and
 * replayed. Points with fewer steps drop out as they finish.
 * The results equal those of running every point alone with twa_run. A point
 * whose `means` is not NULL also gets its per-trajectory window means there.
 *
 * With opts->ws_route = TWA_ROUTE_RESIDENT (precision TWA_PREC_FP32, every
 * N <= TWA_RESIDENT_MAX_N) the whole scan is one launch per CTA shape: each CTA
 * integrates its trajectories of one point for all of that point's steps with
 * the state in shared memory (results equal each point run alone on that
 * route; tiles receives (0, 0)).
 *
 * Tile shapes: unless TWA_TC_BN / TWA_TC_KC are set in the environment, a
 * built-in autotuner times the compiled configurations on a few steps of the
 * points that run in the stage with the most work (steps x N^2 of the points
 * still running; the state is saved and restored around the trials) and keeps
 * the fastest. tiles: NULL or int[2] receiving the chosen (BN, K-stage config:
 * 0 = 64-wide stages of four operand images, 1 = 32-wide stages of four
 * images, 3 = 32-wide stages of one operand image and 4 = 64-wide stages of
 * one operand image, the last two for the precisions with at most two products
 * per entry). With 256-wide tiles the BF16 precisions run on CTA pairs (two
 * CTAs of a cluster share each 256-row tile; TWA_TC_PAIR=0 turns this off);
 * every configuration gives the same results bit for bit.
 * Errors: TWA_EINVAL, TWA_EUNSUPPORTED (a precision other than BF16, BF16X3,
 * BF16X2, BF16L2 and BF16B), plus those of twa_init and twa_sync. Synchronises. */
TWA_API int twa_batch_run(const twa_point* pts, int n, int64_t M, uint64_t seed, const twa_opts* opts,
                          twa_obs* out, int* tiles);

/* request of twa_correlation */
typedef struct twa_corr_req {
    int64_t M;              /* trajectories (Philox indices traj_offset + 0 .. M-1),
                               each integrated as three copies                      */
    int64_t prep_steps;     /* steps from the discrete-Wigner start to the kick      */
    int64_t lag_steps;      /* steps after the kick                                  */
    int64_t lag_stride;     /* C(tau) recorded at tau = k lag_stride dt, k = 0 ..
                               lag_steps / lag_stride (k = 0: right after the kick)  */
    double  eps;            /* kick strength in (0, 1): every spin of a copy is
                               rotated by the angle 2 eps                            */
    int64_t n_omega;        /* spectrum points, omega_j = -omega_max + j 2 omega_max
                               / (n_omega - 1), j < n_omega (>= 3)                   */
    double  omega_max;      /* > 0                                                   */
} twa_corr_req;

typedef struct twa_corr_out {
    int64_t M;              /* trajectories                                          */
    int64_t n_lags;         /* 1 + lag_steps / lag_stride                            */
    double  dtau;           /* lag_stride dt                                         */
    double  fwhm, fwhm_se;  /* linewidth: FWHM of S(omega), block-jackknife SE      */
    double  omega_peak;     /* grid frequency of the maximum of S                    */
    double  S_peak;         /* that maximum                                          */
    double  spsm_tau0;      /* Re C(0): the equal-time <S+S-> at the kick            */
} twa_corr_out;

/* Two-time correlation <S+(tau) S-(0)>, its spectrum and the linewidth (Sec.
 * S1, closing part; main text, "Observables and method": S(omega) = 2 Re int
 * dt e^{i omega t} <S+(t) S-(0)>, linewidth = its full width at half maximum).
 *
 * Runs its own M trajectories with the context's parameters, seed, options and
 * precision (the trajectories twa_run would produce; the state of twa_run is
 * neither read nor changed): prep_steps steps, then every trajectory gets two
 * more copies with the same noise (same Philox counters), kicked by
 * eps delta(t) S^x and by eps delta(t) S^y -- every spin rotated about x, resp.
 * y, by 2 eps, the action of exp(-i eps S^b) on Pauli spins -- and the three
 * copies run lag_steps more steps. At lag 0 and every lag_stride-th step the
 * per-trajectory products S^a(t) S^b(t0) and the responses
 * chi_ab = (S^a of the copy kicked by S^b - S^a) / eps (a, b in {x, y}) are
 * summed, and
 *   C(tau) = 1/4 [S^x S^x + S^y S^y + i (S^y S^x - S^x S^y)](tau)
 *          + i/8 (chi_xx + chi_yy + i chi_yx - i chi_xy)(tau)
 * (with S^+ = (S^x + i S^y) / 2, sigma^+ = (sigma^x + i sigma^y) / 2; the
 * commutator part is normalised so that C(0+) = A + <S^z>/2, the equal-time
 * estimator). S(omega) = 2 Re sum_k c_k e^{i omega tau_k} C(tau_k) dtau with
 * trapezoid weights c_k; FWHM from the grid maximum and the linear
 * interpolation of the first half-maximum crossing on each side (NaN if a side
 * has none). Standard errors by delete-one jackknife over min(32, M) blocks of
 * trajectories, the whole estimate recomputed per block. FP64 reductions.
 *
 * C: NULL or host [n_lags][2] (Re, Im of C(tau)); S: NULL or host [n_omega];
 * parts: NULL or host [n_lags][8], the ensemble means of S^x(t)S^x(t0),
 * S^y(t)S^y(t0), S^x(t)S^y(t0), S^y(t)S^x(t0), chi_xx, chi_yx, chi_xy, chi_yy;
 * C_se: NULL or host [n_lags][2], jackknife SE of Re C and Im C. Synchronises.
 * Temporarily holds three contexts' buffers (pump matrix and factor included).
 * Errors: TWA_EINVAL (NULL, bad counts, eps, omega grid), TWA_ENOMEM,
 * TWA_ECUDA, TWA_ENONFINITE, TWA_ETIMEOUT. */
TWA_API int twa_correlation(twa_ctx* ctx, const twa_corr_req* req, twa_corr_out* out, double* C, double* S,
                            double* parts, double* C_se);

/* Ensemble reduction alone: observables and standard errors (the same FP64
 * device reduction twa_observables uses) of M caller-supplied per-trajectory
 * window means, `means` a host array [M][5] in the twa_get_moments order. Used
 * to merge the shards of an ensemble run on several devices. Fills the first
 * block of *out (Sz .. g2_se, M, samples = 1); diagnostics are zero.
 * Errors: TWA_EINVAL (NULL, M < 1), TWA_ENOMEM, TWA_ECUDA. */
TWA_API int twa_reduce_moments(const double* means, int64_t M, int64_t N, twa_obs* out);

/* Largest M that twa_reduce_moments_noalloc accepts. */
#define TWA_NOALLOC_MAX_M 65536

/* Allocation-free variant of twa_reduce_moments, for callers that cannot call
 * cudaMalloc or any allocating routine: code that runs inside a host
 * application whose memory manager owns the whole device (a framework's pool
 * that has reserved it, or a strict memory budget), and latency-critical loops
 * whose policy forbids allocation after start-up. The paper has no counterpart;
 * this is an engineering variant of the same ensemble reduction.
 *
 * Arguments, layout and result are those of twa_reduce_moments (host `means`
 * [M][5], host *out). Instead of device buffers from cudaMalloc it stages the
 * means, the sample count and the results in one file-scope __device__ array of
 * 16 + 5 * TWA_NOALLOC_MAX_M doubles (about 2.6 MB), which every GPU that loads
 * libtwa holds until the process exits.
 *  - Every call looks up that array's device address (cudaGetSymbolAddress) in
 *    the CUDA context current on the calling thread, so it stays right after
 *    cudaDeviceReset and in a context the caller created. The first call in a
 *    context also loads the library's device code into it; make that first
 *    call before any stream capture.
 *  - Work runs on the legacy default stream with synchronous copies, and the
 *    call returns once the results are on the host. So each call synchronises
 *    with every blocking stream of the device, and no call may overlap a
 *    stream capture in cudaStreamCaptureModeGlobal on any thread (that capture
 *    would be invalidated, or the call would fail). It calls no cudaMalloc,
 *    cudaFree or other allocating routine.
 *  - Every call on a device shares the one array and rewrites the count, the
 *    means and the results it uses; calls that overlap on the GPU (from several
 *    host threads) race and must be serialised by the caller.
 * Errors: TWA_EINVAL (NULL, M < 1, N < 1, M > TWA_NOALLOC_MAX_M), TWA_ECUDA. */
TWA_API int twa_reduce_moments_noalloc(const double* means, int64_t M, int64_t N, twa_obs* out);

/* Check of the device-side timeout path, without any fault (the paper has no
 * counterpart). Enqueues on the context's stream one bounded wait -- the
 * routine every tensor-core kernel uses on its shared-memory mbarriers -- on a
 * barrier that nothing completes, with a limit of limit_us microseconds. The
 * wait gives up, records a timeout on the context and returns; the next call
 * that synchronises (twa_sync, twa_observables, ...) returns TWA_ETIMEOUT, as it
 * would after a real wait ran out. The record stays: such a context should be
 * destroyed. Errors: TWA_EINVAL (NULL, limit_us outside [1, 10^7]). */
TWA_API int twa_wait_probe(twa_ctx* ctx, int64_t limit_us);

/* Start (enable = 1) or stop (0) timing every kernel the context launches with
 * a pair of CUDA events recorded on its stream around the launch. Recording
 * adds no synchronisation. Errors: TWA_EINVAL. */
TWA_API int twa_profile(twa_ctx* ctx, int enable);

/* Synchronise, then return per kernel class (TWA_PROF_*), summed over the
 * launches since profiling started, the event time in ms, the number of
 * launches, and for the dense mixed-precision contractions (0 for other
 * classes) two FLOP counts: `flops`, the tensor-core FLOPs issued -- 2 x the
 * multiply-adds over all of W and the lower triangle of L times the products
 * per entry, plus the second product over the K stages of the two-product band
 * (TWA_PREC_BF16L2, TWA_PREC_BF16B) -- and `alg_flops`, the algorithmic count:
 * 2 x the multiply-adds of the defined products over their nonzero entries,
 * counted once whatever the precision. Then clear the record. Each array holds
 * TWA_PROF_KINDS entries and may be NULL. */
TWA_API int twa_profile_read(twa_ctx* ctx, double* ms, int64_t* launches, double* flops, double* alg_flops);

/* One-line description of the last error on ctx (or of the last failed
 * twa_init when ctx is NULL). Never NULL. */
TWA_API const char* twa_last_error(const twa_ctx* ctx);

/* Free the context and all device memory it owns. NULL is allowed. */
TWA_API void twa_destroy(twa_ctx* ctx);

/* Library version string. */
TWA_API const char* twa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TWA_H */

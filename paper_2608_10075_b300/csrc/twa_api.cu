// C-ABI entry points of libtwa (declared and documented in include/twa.h).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>

#include "twa_internal.cuh"


namespace twa {

cudaError_t dev_malloc(twa_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    if (c && c->opts.alloc && c->opts.free) {
        *p = c->opts.alloc(bytes, (void*)c->stream, c->opts.alloc_user);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

void dev_free(twa_ctx* c, void* p) {
    if (!p) return;
    if (c && c->opts.alloc && c->opts.free) c->opts.free(p, (void*)c->stream, c->opts.alloc_user);
    else cudaFree(p);
}

cudaError_t dev_malloc_async(twa_ctx* c, void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    if (c && c->opts.alloc && c->opts.free) {
        *p = c->opts.alloc(bytes, (void*)st, c->opts.alloc_user);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

void dev_free_async(twa_ctx* c, void* p, cudaStream_t st) {
    if (!p) return;
    if (c && c->opts.alloc && c->opts.free) c->opts.free(p, (void*)st, c->opts.alloc_user);
    else cudaFreeAsync(p, st);
}

}  // namespace twa

namespace {
thread_local std::string g_init_error;
constexpr int64_t MAX_N = 60000;          // W and L in FP64 take 2 N^2 8 B (57.6 GB at the limit)
constexpr int64_t MAX_COUNTER = 0xFFFFFFFFll;

bool use_tc(const twa_ctx* c) { return c->opts.precision != TWA_PREC_FP64; }
}  // namespace

namespace twa {

int set_error(twa_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_init_error = msg;
    return code;
}

int cuda_check(twa_ctx* c, cudaError_t e, const char* what) {
    return set_error(c, e == cudaErrorMemoryAllocation ? TWA_ENOMEM : TWA_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace twa

using twa::set_error;

namespace {

__global__ void k_window_means(const double* mom, const int64_t* cnt, double* out, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) out[e] = mom[e] / (double)(*cnt);
}

int free_run_buffers(twa_ctx* c) {
    twa::f64_free(c);
    if (c->tc) twa::tc_free_run(c);
    twa::dev_free(c, c->mom);
    c->mom = nullptr;
    return TWA_OK;
}

// Fix M, allocate the trajectory buffers and zero the window sums.
int fix_M(twa_ctx* c, int64_t M) {
    c->M = M;
    if (twa::dev_malloc(c, &c->mom, sizeof(double) * 5 * M) != cudaSuccess) {
        c->M = 0;
        return set_error(c, TWA_ENOMEM, "device window sums");
    }
    TWA_CUDA(c, cudaMemsetAsync(c->mom, 0, sizeof(double) * 5 * M, c->stream));
    int rc = use_tc(c) ? twa::tc_alloc(c) : twa::f64_alloc(c);
    if (rc) {
        free_run_buffers(c);
        c->M = 0;
    }
    return rc;
}

int run_eager(twa_ctx* c, int64_t t0, int64_t steps) {
    return use_tc(c) ? twa::tc_run(c, t0, steps) : twa::f64_run(c, steps);
}

// Capture step t on a private stream into the graph of its parity. The step's
// kernels read the step counter from device memory, so one graph serves every
// step of that parity (the dense mixed-precision step alternates two buffers).
int capture_step(twa_ctx* c, int64_t t) {
    if (!c->capture_stream) TWA_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    cudaStream_t saved = c->stream;
    c->stream = c->capture_stream;
    cudaGraph_t g = nullptr;
    int rc = TWA_OK;
    if (cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = TWA_ECUDA;
    } else {
        rc = use_tc(c) ? twa::tc_launch_step(c, t) : twa::f64_run(c, 1);
        if (cudaStreamEndCapture(c->capture_stream, &g) != cudaSuccess) rc = TWA_ECUDA;
    }
    c->stream = saved;
    cudaGraphExec_t& slot = c->step_graph[t & 1];
    if (rc == TWA_OK && g && cudaGraphInstantiate(&slot, g, 0) != cudaSuccess) {
        slot = nullptr;
        rc = TWA_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();   // a failed capture leaves nothing pending: steps then run eagerly
    return rc;
}

void drop_graphs(twa_ctx* c) {
    for (auto& g : c->step_graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Steps either replay the captured step graphs or launch the kernels directly
// (profiling, very short runs, or TWA_NO_GRAPH set).
int run_steps(twa_ctx* c, int64_t steps) {
    if (c->res_W || c->res_tc) return twa::res_run(c, steps);   // resident route: all steps in one launch
    int64_t t = c->steps;
    if (c->profiling || steps < 4 || c->graph_failed || getenv("TWA_NO_GRAPH")) return run_eager(c, t, steps);
    int rc;
    if (!c->step_graph[0]) {
        if ((rc = run_eager(c, t, 1))) return rc;   // first launches set kernel attributes outside any capture
        ++t;
        --steps;
        if (capture_step(c, t) != TWA_OK || capture_step(c, t + 1) != TWA_OK) {
            drop_graphs(c);
            c->graph_failed = true;
            return run_eager(c, t, steps);
        }
    }
    if (use_tc(c) && (rc = twa::tc_prime(c, t))) return rc;
    for (int64_t s = 0; s < steps; ++s) TWA_CUDA(c, cudaGraphLaunch(c->step_graph[(t + s) & 1], c->stream));
    if (use_tc(c)) twa::tc_steps_done(c, t + steps);
    return TWA_OK;
}

int check_device_flags(twa_ctx* c) {
    unsigned long long fl[twa::FLAG_COUNT];
    TWA_CUDA(c, cudaStreamSynchronize(c->stream));
    TWA_CUDA(c, cudaMemcpy(fl, c->d_flags, sizeof(fl), cudaMemcpyDeviceToHost));
    if (fl[twa::FLAG_TIMEOUT])
        return set_error(c, TWA_ETIMEOUT,
                         "a device-side wait ran out of its time limit (" + std::to_string(fl[twa::FLAG_TIMEOUT]) +
                             " waits)");
    if (fl[twa::FLAG_NONFINITE])
        return set_error(c, TWA_ENONFINITE,
                         std::to_string(fl[twa::FLAG_NONFINITE]) + " spin updates produced NaN/Inf");
    return TWA_OK;
}

}  // namespace

extern "C" {

const char* twa_version(void) { return "libtwa 0.1 (sm_103a)"; }

int twa_opts_default(twa_opts* o) {
    if (!o) return TWA_EINVAL;
    memset(o, 0, sizeof(*o));
    o->precision = TWA_PREC_FP64;
    o->init_state = -1;
    o->window_start = 0.0;
    o->renormalize = 1;
    o->clip_negative = 0;
    o->stream = nullptr;
    o->sample_stride = 1;
    return TWA_OK;
}

int twa_init(twa_ctx** out, int64_t N, double alpha, double w, double Gamma, double dt, uint64_t seed,
             const twa_opts* opts) {
    twa::NvtxRange range("twa_init");
    if (!out) return set_error(nullptr, TWA_EINVAL, "twa_init: out is NULL");
    *out = nullptr;
    twa_opts o;
    twa_opts_default(&o);
    if (opts) o = *opts;
    if (N < 1 || N > MAX_N) return set_error(nullptr, TWA_EINVAL, "twa_init: N must be in [1, 60000]");
    if (!(alpha >= 0.0)) return set_error(nullptr, TWA_EINVAL, "twa_init: alpha must be >= 0 (or +INF)");
    if (!(w >= 0.0) || isinf(w)) return set_error(nullptr, TWA_EINVAL, "twa_init: w must be finite and >= 0");
    if (!(Gamma >= 0.0) || isinf(Gamma)) return set_error(nullptr, TWA_EINVAL, "twa_init: Gamma must be finite and >= 0");
    if (!(dt > 0.0) || isinf(dt)) return set_error(nullptr, TWA_EINVAL, "twa_init: dt must be finite and > 0");
    if (o.precision < TWA_PREC_FP64 || o.precision > TWA_PREC_BF16B)
        return set_error(nullptr, TWA_EINVAL, "twa_init: unknown precision");
    if (o.init_state != -1 && o.init_state != 1) return set_error(nullptr, TWA_EINVAL, "twa_init: init_state must be +-1");
    if (!(o.window_start >= 0.0) || isinf(o.window_start))
        return set_error(nullptr, TWA_EINVAL, "twa_init: window_start must be finite and >= 0");
    if (o.traj_offset < 0 || o.traj_offset > MAX_COUNTER)
        return set_error(nullptr, TWA_EINVAL, "twa_init: traj_offset must be in [0, 2^32-1]");
    if (o.ws_route != TWA_ROUTE_DENSE && o.ws_route != TWA_ROUTE_FFT && o.ws_route != TWA_ROUTE_RESIDENT)
        return set_error(nullptr, TWA_EINVAL,
                         "twa_init: ws_route must be TWA_ROUTE_DENSE, TWA_ROUTE_FFT or TWA_ROUTE_RESIDENT");
    if (o.ws_route == TWA_ROUTE_RESIDENT && o.precision != TWA_PREC_FP32 && o.precision != TWA_PREC_BF16X2)
        return set_error(nullptr, TWA_EUNSUPPORTED,
                         "twa_init: the resident route runs with precision TWA_PREC_FP32 or TWA_PREC_BF16X2");
    if (o.ws_route == TWA_ROUTE_RESIDENT && N > TWA_RESIDENT_MAX_N)
        return set_error(nullptr, TWA_EUNSUPPORTED, "twa_init: the resident route holds N <= 512 sites");
    if (o.ws_route == TWA_ROUTE_RESIDENT && o.precision == TWA_PREC_BF16X2 && N > TWA_RESIDENT_TC_MAX_N)
        return set_error(nullptr, TWA_EUNSUPPORTED,
                         "twa_init: the tensor-core resident route (TWA_PREC_BF16X2) holds N <= 128 sites");
    if (o.ws_route == TWA_ROUTE_FFT && o.precision == TWA_PREC_FP64)
        return set_error(nullptr, TWA_EUNSUPPORTED, "twa_init: the FFT route runs with the tensor-core precisions only");
    if ((o.alloc == nullptr) != (o.free == nullptr))
        return set_error(nullptr, TWA_EINVAL, "twa_init: give both alloc and free, or neither");
    if (o.sample_stride < 0 || o.sample_stride > MAX_COUNTER)
        return set_error(nullptr, TWA_EINVAL, "twa_init: sample_stride must be in [0, 2^32-1]");
    if (o.integrator != TWA_INT_HEUN && o.integrator != TWA_INT_MIDPOINT)
        return set_error(nullptr, TWA_EINVAL, "twa_init: integrator must be TWA_INT_HEUN or TWA_INT_MIDPOINT");
    if (o.noise_route != TWA_NOISE_CHOLESKY && o.noise_route != TWA_NOISE_CIRCULANT)
        return set_error(nullptr, TWA_EINVAL, "twa_init: noise_route must be TWA_NOISE_CHOLESKY or TWA_NOISE_CIRCULANT");
    if (o.noise_route == TWA_NOISE_CIRCULANT && o.ws_route != TWA_ROUTE_FFT)
        return set_error(nullptr, TWA_EUNSUPPORTED, "twa_init: the circulant noise draw needs ws_route = TWA_ROUTE_FFT");

    twa_ctx* c = new (std::nothrow) twa_ctx();
    if (!c) return set_error(nullptr, TWA_ENOMEM, "twa_init: host allocation failed");
    c->N = N;
    c->alpha = alpha;
    c->w = w;
    c->Gamma = Gamma;
    c->dt = dt;
    c->seed = seed;
    c->opts = o;
    c->stream = (cudaStream_t)o.stream;
    c->n_window = (int64_t)floor(o.window_start / dt + 0.5);
    c->n_stride = o.sample_stride > 1 ? o.sample_stride : 1;
    int rc = TWA_OK;
    auto fail = [&](int code) {
        g_init_error = c->err;
        twa_destroy(c);
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        twa::cuda_check(c, e, "cudaGetDevice");
        return fail(TWA_ECUDA);
    }
    if (twa::dev_malloc(c, &c->W64, sizeof(double) * N * N) != cudaSuccess ||
        twa::dev_malloc(c, &c->L64, sizeof(double) * N * N) != cudaSuccess ||
        twa::dev_malloc(c, &c->d_t, sizeof(int64_t)) != cudaSuccess ||
        twa::dev_malloc(c, &c->d_count, sizeof(int64_t)) != cudaSuccess ||
        twa::dev_malloc(c, &c->d_flags, sizeof(unsigned long long) * twa::FLAG_COUNT) != cudaSuccess) {
        set_error(c, TWA_ENOMEM, "twa_init: device allocation failed");
        return fail(TWA_ENOMEM);
    }
    if (cudaMemsetAsync(c->d_t, 0, sizeof(int64_t), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_count, 0, sizeof(int64_t), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned long long) * twa::FLAG_COUNT, c->stream) != cudaSuccess) {
        set_error(c, TWA_ECUDA, "twa_init: cudaMemsetAsync failed");
        return fail(TWA_ECUDA);
    }
    {
        twa::NvtxRange r1("twa_init: pump matrix, Cholesky factor, spectrum");
        if ((rc = twa::setup_pump(c))) return fail(rc);
    }
    {
        twa::NvtxRange r2("twa_init: operand images, FFT plan");
        if (use_tc(c) && (rc = twa::tc_prepare(c))) return fail(rc);
        if (o.ws_route == TWA_ROUTE_FFT && (rc = twa::fft_prepare(c))) return fail(rc);
        if (o.ws_route == TWA_ROUTE_RESIDENT && (rc = twa::res_prepare(c))) return fail(rc);
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        twa::cuda_check(c, e, "twa_init");
        return fail(TWA_ECUDA);
    }
    *out = c;
    return TWA_OK;
}

int twa_run(twa_ctx* c, int64_t M, int64_t steps) {
    twa::NvtxRange range("twa_run: step block");
    if (!c) return set_error(nullptr, TWA_EINVAL, "twa_run: ctx is NULL");
    if (M < 1 || M > (int64_t)1 << 30) return set_error(c, TWA_EINVAL, "twa_run: M must be in [1, 2^30]");
    if (steps < 0) return set_error(c, TWA_EINVAL, "twa_run: steps must be >= 0");
    if (c->M != 0 && M != c->M)
        return set_error(c, TWA_EINVAL, "twa_run: M differs from the trajectory count fixed by the first call");
    if (c->steps + steps > MAX_COUNTER) return set_error(c, TWA_EINVAL, "twa_run: step counter would exceed 2^32-1");
    if (c->opts.traj_offset + M - 1 > MAX_COUNTER)
        return set_error(c, TWA_EINVAL, "twa_run: traj_offset + M exceeds the 32-bit trajectory counter");
    int rc;
    if (c->M == 0) {
        if ((rc = fix_M(c, M))) return rc;
        rc = use_tc(c) ? twa::tc_init_state(c) : twa::f64_init_state(c);
        if (rc) return rc;
    }
    if (steps == 0) return TWA_OK;
    if ((rc = run_steps(c, steps))) return rc;
    c->steps += steps;
    return TWA_OK;
}

int twa_sync(twa_ctx* c) {
    if (!c) return set_error(nullptr, TWA_EINVAL, "twa_sync: ctx is NULL");
    return check_device_flags(c);
}

int twa_observables(twa_ctx* c, twa_obs* out) {
    twa::NvtxRange range("twa_observables: ensemble reduction");
    if (!c || !out) return set_error(c, TWA_EINVAL, "twa_observables: NULL argument");
    if (c->M == 0) return set_error(c, TWA_ESTATE, "twa_observables: no trajectories yet");
    int rc = check_device_flags(c);
    if (rc) return rc;
    int64_t cnt = 0;
    TWA_CUDA(c, cudaMemcpy(&cnt, c->d_count, sizeof(cnt), cudaMemcpyDeviceToHost));
    if (cnt == 0) return set_error(c, TWA_ESTATE, "twa_observables: no step inside the averaging window yet");
    memset(out, 0, sizeof(*out));
    if ((rc = twa::reduce_observables(c, out))) return rc;
    out->M = c->M;
    out->steps = c->steps;
    out->w_max = c->w_max;
    out->w_min = c->w_min;
    out->w_tilde = (c->Gamma > 0) ? c->w_max / (c->Gamma * (double)c->N) : INFINITY;
    out->stability = fmax(c->Gamma * (double)c->N, c->w_max) * c->dt;
    out->min_pivot = c->min_pivot;
    out->clipped = c->clipped;
    out->factor_residual = c->factor_residual;
    out->fft_length = c->fft ? c->fft->P : 0;
    out->fft_ctas = c->fft ? c->fft->C : 0;
    unsigned long long fl[twa::FLAG_COUNT];
    TWA_CUDA(c, cudaMemcpy(fl, c->d_flags, sizeof(fl), cudaMemcpyDeviceToHost));
    out->nonfinite = (int64_t)fl[twa::FLAG_NONFINITE];
    return TWA_OK;
}

int twa_get_state(twa_ctx* c, double* sx, double* sy, double* sz, int on_device) {
    if (!c || !sx || !sy || !sz) return set_error(c, TWA_EINVAL, "twa_get_state: NULL argument");
    if (c->M == 0) return set_error(c, TWA_ESTATE, "twa_get_state: no trajectories yet");
    const int64_t M = c->M, N = c->N;
    const size_t row = sizeof(double) * N;
    if (use_tc(c)) {
        double *dx = sx, *dy = sy, *dz = sz;
        twa::Scratch<double> tmp_buf(c, c->stream);
        if (!on_device) {
            TWA_CUDA(c, tmp_buf.alloc(3 * row * M));
            double* tmp = tmp_buf.p;
            dx = tmp;
            dy = tmp + M * N;
            dz = tmp + 2 * M * N;
        }
        int rc = twa::tc_get_state(c, dx, dy, dz);
        if (rc) return rc;
        if (!on_device) {
            TWA_CUDA(c, cudaMemcpyAsync(sx, dx, row * M, cudaMemcpyDeviceToHost, c->stream));
            TWA_CUDA(c, cudaMemcpyAsync(sy, dy, row * M, cudaMemcpyDeviceToHost, c->stream));
            TWA_CUDA(c, cudaMemcpyAsync(sz, dz, row * M, cudaMemcpyDeviceToHost, c->stream));
        }
    } else {
        const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        TWA_CUDA(c, cudaMemcpy2DAsync(sx, row, c->xy, 2 * row, row, M, k, c->stream));
        TWA_CUDA(c, cudaMemcpy2DAsync(sy, row, c->xy + N, 2 * row, row, M, k, c->stream));
        TWA_CUDA(c, cudaMemcpyAsync(sz, c->z, row * M, k, c->stream));
    }
    return check_device_flags(c);
}

int twa_set_state(twa_ctx* c, int64_t M, const double* sx, const double* sy, const double* sz, int on_device) {
    if (!c || !sx || !sy || !sz) return set_error(c, TWA_EINVAL, "twa_set_state: NULL argument");
    if (M < 1 || M > (int64_t)1 << 30) return set_error(c, TWA_EINVAL, "twa_set_state: M must be in [1, 2^30]");
    if (c->M != 0 && M != c->M) return set_error(c, TWA_EINVAL, "twa_set_state: M differs from the fixed M");
    int rc;
    if (c->M == 0 && (rc = fix_M(c, M))) return rc;
    const int64_t N = c->N;
    const size_t row = sizeof(double) * N;
    if (use_tc(c)) {
        const double *dx = sx, *dy = sy, *dz = sz;
        twa::Scratch<double> tmp_buf(c, c->stream);
        if (!on_device) {
            TWA_CUDA(c, tmp_buf.alloc(3 * row * M));
            double* tmp = tmp_buf.p;
            TWA_CUDA(c, cudaMemcpyAsync(tmp, sx, row * M, cudaMemcpyHostToDevice, c->stream));
            TWA_CUDA(c, cudaMemcpyAsync(tmp + M * N, sy, row * M, cudaMemcpyHostToDevice, c->stream));
            TWA_CUDA(c, cudaMemcpyAsync(tmp + 2 * M * N, sz, row * M, cudaMemcpyHostToDevice, c->stream));
            dx = tmp;
            dy = tmp + M * N;
            dz = tmp + 2 * M * N;
        }
        rc = twa::tc_set_state(c, dx, dy, dz);
        if (rc) return rc;
    } else {
        const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        TWA_CUDA(c, cudaMemcpy2DAsync(c->xy, 2 * row, sx, row, row, M, k, c->stream));
        TWA_CUDA(c, cudaMemcpy2DAsync(c->xy + N, 2 * row, sy, row, row, M, k, c->stream));
        TWA_CUDA(c, cudaMemcpyAsync(c->z, sz, row * M, k, c->stream));
        if ((rc = twa::f64_state_changed(c))) return rc;
    }
    if (!on_device) TWA_CUDA(c, cudaStreamSynchronize(c->stream));
    return TWA_OK;
}

int twa_get_state_f32(twa_ctx* c, float* sx, float* sy, float* sz, int on_device) {
    if (!c || !sx || !sy || !sz) return set_error(c, TWA_EINVAL, "twa_get_state_f32: NULL argument");
    if (c->M == 0) return set_error(c, TWA_ESTATE, "twa_get_state_f32: no trajectories yet");
    if (!use_tc(c)) return set_error(c, TWA_EUNSUPPORTED, "twa_get_state_f32: the FP64 path keeps FP64 spins");
    const size_t bytes = sizeof(float) * (size_t)c->M * c->N;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    twa::TcState* t = c->tc;
    TWA_CUDA(c, cudaMemcpyAsync(sx, t->X, bytes, k, c->stream));
    TWA_CUDA(c, cudaMemcpyAsync(sy, t->Y, bytes, k, c->stream));
    TWA_CUDA(c, cudaMemcpyAsync(sz, t->Z, bytes, k, c->stream));
    return check_device_flags(c);
}

int twa_set_state_f32(twa_ctx* c, int64_t M, const float* sx, const float* sy, const float* sz, int on_device) {
    if (!c || !sx || !sy || !sz) return set_error(c, TWA_EINVAL, "twa_set_state_f32: NULL argument");
    if (M < 1 || M > (int64_t)1 << 30) return set_error(c, TWA_EINVAL, "twa_set_state_f32: M must be in [1, 2^30]");
    if (c->M != 0 && M != c->M) return set_error(c, TWA_EINVAL, "twa_set_state_f32: M differs from the fixed M");
    if (!use_tc(c)) return set_error(c, TWA_EUNSUPPORTED, "twa_set_state_f32: the FP64 path keeps FP64 spins");
    int rc;
    if (c->M == 0 && (rc = fix_M(c, M))) return rc;
    // straight into the FP32 state the mixed-precision step works on
    const size_t bytes = sizeof(float) * (size_t)M * c->N;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    twa::TcState* t = c->tc;
    TWA_CUDA(c, cudaMemcpyAsync(t->X, sx, bytes, k, c->stream));
    TWA_CUDA(c, cudaMemcpyAsync(t->Y, sy, bytes, k, c->stream));
    TWA_CUDA(c, cudaMemcpyAsync(t->Z, sz, bytes, k, c->stream));
    if ((rc = twa::tc_state_changed(c))) return rc;
    if (!on_device) TWA_CUDA(c, cudaStreamSynchronize(c->stream));
    return TWA_OK;
}

int twa_get_moments(twa_ctx* c, double* out, int on_device) {
    if (!c || !out) return set_error(c, TWA_EINVAL, "twa_get_moments: NULL argument");
    if (c->M == 0) return set_error(c, TWA_ESTATE, "twa_get_moments: no trajectories yet");
    int64_t cnt = 0;
    TWA_CUDA(c, cudaMemcpyAsync(&cnt, c->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    TWA_CUDA(c, cudaStreamSynchronize(c->stream));
    if (cnt == 0) return set_error(c, TWA_ESTATE, "twa_get_moments: no step inside the averaging window yet");
    const int64_t n = 5 * c->M;
    double* dst = out;
    twa::Scratch<double> dst_buf(c, c->stream);
    if (!on_device) {
        TWA_CUDA(c, dst_buf.alloc(sizeof(double) * n));
        dst = dst_buf.p;
    }
    k_window_means<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->mom, c->d_count, dst, n);
    TWA_CUDA(c, cudaGetLastError());
    if (!on_device) {
        TWA_CUDA(c, cudaMemcpyAsync(out, dst, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    }
    return check_device_flags(c);
}

int twa_field(twa_ctx* c, const double* s, double* P, int64_t K) {
    if (!c || !s || !P) return set_error(c, TWA_EINVAL, "twa_field: NULL argument");
    if (K < 1 || K > (int64_t)1 << 30) return set_error(c, TWA_EINVAL, "twa_field: K must be in [1, 2^30]");
    return use_tc(c) ? twa::tc_field(c, s, P, K) : twa::f64_field(c, s, P, K);
}

int twa_contract(twa_ctx* c, int matrix, const double* s, double* P, int64_t K) {
    if (!c || !s || !P) return set_error(c, TWA_EINVAL, "twa_contract: NULL argument");
    if (matrix != TWA_MAT_W && matrix != TWA_MAT_L)
        return set_error(c, TWA_EINVAL, "twa_contract: matrix must be TWA_MAT_W or TWA_MAT_L");
    if (K < 1 || K > (int64_t)1 << 30) return set_error(c, TWA_EINVAL, "twa_contract: K must be in [1, 2^30]");
    const int which = matrix == TWA_MAT_L ? 1 : 0;
    return use_tc(c) ? twa::tc_field(c, s, P, K, which) : twa::f64_field(c, s, P, K, which);
}

int twa_grad(twa_ctx* c, const twa_grad_req* r, twa_grad_out* out, double* per_traj) {
    twa::NvtxRange range("twa_grad: forward with checkpoints, reverse sweep");
    if (!c || !r || !out) return set_error(c, TWA_EINVAL, "twa_grad: NULL argument");
    if (r->objective != TWA_OBJ_SPSM && r->objective != TWA_OBJ_G2)
        return set_error(c, TWA_EINVAL, "twa_grad: unknown objective");
    if (r->M < 1 || r->M > (int64_t)1 << 30) return set_error(c, TWA_EINVAL, "twa_grad: M must be in [1, 2^30]");
    if (r->steps < 1 || r->steps > MAX_COUNTER) return set_error(c, TWA_EINVAL, "twa_grad: steps must be in [1, 2^32-1]");
    if (c->opts.traj_offset + r->M - 1 > MAX_COUNTER)
        return set_error(c, TWA_EINVAL, "twa_grad: traj_offset + M exceeds the 32-bit trajectory counter");
    if (!(c->w > 0.0)) return set_error(c, TWA_EUNSUPPORTED, "twa_grad: needs w > 0");
    if (c->opts.precision == TWA_PREC_TF32 || c->opts.precision == TWA_PREC_FP32)
        return set_error(c, TWA_EUNSUPPORTED, "twa_grad: runs on the FP64 and BF16 precisions (BF16, BF16X3, BF16X2, BF16L2, BF16B)");
    if (c->opts.integrator != TWA_INT_HEUN)
        return set_error(c, TWA_EUNSUPPORTED, "twa_grad: differentiates the Heun integrator only");
    if (c->opts.noise_route != TWA_NOISE_CHOLESKY)
        return set_error(c, TWA_EUNSUPPORTED, "twa_grad: differentiates the Cholesky noise draw only");
    if (r->want_alpha && (c->alpha == 0.0 || isinf(c->alpha)))
        return set_error(c, TWA_EUNSUPPORTED, "twa_grad: d/dalpha needs 0 < alpha < inf");
    memset(out, 0, sizeof(*out));
    int rc = twa::grad(c, r, out, per_traj);
    if (rc) return rc;
    return check_device_flags(c);
}

int twa_reduce_moments(const double* means, int64_t M, int64_t N, twa_obs* out) {
    twa::NvtxRange range("twa_reduce_moments");
    if (!means || !out || M < 1 || N < 1) return set_error(nullptr, TWA_EINVAL, "twa_reduce_moments: bad argument");
    twa_ctx tmp;
    tmp.N = N;
    tmp.M = M;
    int rc = TWA_OK;
    if (cudaMalloc(&tmp.mom, sizeof(double) * 5 * M) != cudaSuccess ||
        cudaMalloc(&tmp.d_count, sizeof(int64_t)) != cudaSuccess) {
        rc = set_error(nullptr, TWA_ENOMEM, "twa_reduce_moments: device allocation failed");
    } else {
        const int64_t one = 1;
        memset(out, 0, sizeof(*out));
        if (cudaMemcpy(tmp.mom, means, sizeof(double) * 5 * M, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(tmp.d_count, &one, sizeof(one), cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = set_error(nullptr, TWA_ECUDA, "twa_reduce_moments: upload failed");
        } else if ((rc = twa::reduce_observables(&tmp, out))) {
            g_init_error = tmp.err;
        }
        out->M = M;
    }
    if (tmp.mom) cudaFree(tmp.mom);
    if (tmp.d_count) cudaFree(tmp.d_count);
    tmp.mom = nullptr;
    tmp.d_count = nullptr;
    return rc;
}

int twa_wait_probe(twa_ctx* c, int64_t limit_us) {
    if (!c) return set_error(nullptr, TWA_EINVAL, "twa_wait_probe: ctx is NULL");
    if (limit_us < 1 || limit_us > 10000000)
        return set_error(c, TWA_EINVAL, "twa_wait_probe: limit_us must be in [1, 10^7]");
    return twa::wait_probe(c, limit_us * 1000);
}

int twa_profile(twa_ctx* c, int enable) {
    if (!c) return set_error(nullptr, TWA_EINVAL, "twa_profile: ctx is NULL");
    c->profiling = enable != 0;
    return TWA_OK;
}

int twa_profile_read(twa_ctx* c, double* ms, int64_t* launches, double* flops, double* alg_flops) {
    if (!c) return set_error(nullptr, TWA_EINVAL, "twa_profile_read: ctx is NULL");
    TWA_CUDA(c, cudaStreamSynchronize(c->stream));
    double t[TWA_PROF_KINDS] = {0}, f[TWA_PROF_KINDS] = {0}, fa[TWA_PROF_KINDS] = {0};
    int64_t n[TWA_PROF_KINDS] = {0};
    int rc = TWA_OK;
    for (auto& r : c->prof) {
        float e = 0.f;
        if (cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) rc = TWA_ECUDA;
        if (r.kind >= 0 && r.kind < TWA_PROF_KINDS) {
            t[r.kind] += e;
            n[r.kind] += 1;
            f[r.kind] += r.flops;
            fa[r.kind] += r.alg;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->prof.clear();
    for (int k = 0; k < TWA_PROF_KINDS; ++k) {
        if (ms) ms[k] = t[k];
        if (launches) launches[k] = n[k];
        if (flops) flops[k] = f[k];
        if (alg_flops) alg_flops[k] = fa[k];
    }
    if (rc) return set_error(c, rc, "twa_profile_read: cudaEventElapsedTime failed");
    return TWA_OK;
}

const char* twa_last_error(const twa_ctx* c) {
    if (!c) return g_init_error.c_str();
    return c->err.c_str();
}

void twa_destroy(twa_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    for (auto& r : c->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    free_run_buffers(c);
    if (c->tc) twa::tc_free(c);
    twa::fft_free(c);
    twa::res_free(c);
    void* p[] = {c->W64, c->L64, c->d_t, c->d_count, c->d_flags};
    for (void* q : p) twa::dev_free(c, q);
    delete c;
}

}  // extern "C"

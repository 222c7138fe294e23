// Resident route (ws_route = TWA_ROUTE_RESIDENT): small systems whose whole run
// fits one launch. Every CTA owns T trajectories of one problem (a context, or
// one point of a batched scan) and integrates them for all steps of the call
// with the state, the predictor and the noise part held in shared memory; W
// and L stay in shared memory for the whole launch when they fit (N <= ~100),
// otherwise they are streamed through it in 32-column chunks from L2. There is
// no communication between CTAs, so a call is one launch however many steps
// it has, and a batch of points of different N is one launch per CTA shape.
//
// Arithmetic: FP32 throughout -- the contractions of Eq. S1 (sum_j w_ij s_j,
// (L eta)_i) as FP32 FMA chains over j, the collective sums in FP32, the
// FP32 Box-Muller normals of the mixed paths (not rounded to BF16), Heun or
// the semi-implicit midpoint scheme with the roundings of the tensor-core
// epilogues, renormalisation to sqrt(3); window moments in FP64.
//
// Shared memory per CTA (floats): S [N][2T] (x, y of the T trajectories at
// site j, column 2t = x, 2t + 1 = y) and Sz [N][T]; the predictor P, Pz in the
// same layout (first the normals eta of the step); the noise part Q [N][2T];
// then either W and L with row pitch N + 1 or one [N][33] chunk buffer.
// Contractions: thread (ti, tc) accumulates rows ti*RI .. ti*RI + RI - 1
// against columns 4 tc .. 4 tc + 3 (trajectories 2 tc and 2 tc + 1), so the
// same thread then applies the integrator's update to exactly those entries.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "twa_internal.cuh"

namespace twa {
namespace {

constexpr int RT = 512;        // threads per CTA
constexpr int RI_MAX = 8;      // rows per thread (at most)
constexpr int KCH = 32;        // K columns of a streamed chunk of W or L
constexpr size_t RES_SMEM_MAX = 215 * 1024;

struct ResProblem {
    const float* W;             // [N][N] FP32
    const float* L;             // [N][N] FP32, lower triangular
    float *X, *Y, *Z;           // state [M][N]
    double* mom;                // window sums [M][5]
    unsigned long long* flags;
    int64_t M, N, m0, t0, steps, n_window, stride;
    uint64_t seed;
    float G, hdt, sgdt, sdt;
    int renorm, integ;
};

// shared-memory floats of a CTA with T trajectories of N sites
__host__ __device__ inline size_t res_state_floats(int64_t N, int T) { return (size_t)8 * N * T; }
__host__ __device__ inline size_t res_matrix_floats(int64_t N, bool resident) {
    return resident ? (size_t)2 * N * (N + 1) : (size_t)N * (KCH + 1);
}

template <int T>
__device__ __forceinline__ void col_sums(const float* xy, const float* z, int64_t N, float* out, bool with_z) {
    // out[c] = sum_j xy[j][c] (c < 2T), out[2T + t] = sum_j z[j][t]; each column
    // by a group of at most 32 consecutive lanes of one warp, FP32, fixed order
    constexpr int G2 = (RT / (2 * T) < 32) ? RT / (2 * T) : 32;
    constexpr int G1 = (RT / T < 32) ? RT / T : 32;
    const int tid = threadIdx.x;
    if (tid < 2 * T * G2) {
        const int c = tid / G2, sub = tid % G2;
        float s = 0.f;
        for (int64_t j = sub; j < N; j += G2) s += xy[j * 2 * T + c];
        for (int o = G2 / 2; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (sub == 0) out[c] = s;
    }
    if (with_z && tid < T * G1) {
        const int c = tid / G1, sub = tid % G1;
        float s = 0.f;
        for (int64_t j = sub; j < N; j += G1) s += z[j * T + c];
        for (int o = G1 / 2; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (sub == 0) out[2 * T + c] = s;
    }
}

// acc[r][k] = sum_j A[i_r][j] V[j][4 tc + k], i_r = ti RI + r. TRI: A is lower
// triangular, so the sum stops at the thread's last row.
template <int T, bool RES, bool TRI>
__device__ __forceinline__ void contract(const float* A_glob, const float* A_res, float* stage, const float* V,
                                         int64_t N, int RI, int ti, int tc, float (&acc)[RI_MAX][4]) {
#pragma unroll
    for (int r = 0; r < RI_MAX; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[r][k] = 0.f;
    const int64_t i0 = (int64_t)ti * RI;
    const int64_t jmax = TRI ? (i0 + RI < N ? i0 + RI : N) : N;
    if constexpr (RES) {
        for (int64_t j = 0; j < jmax; ++j) {
            const float4 b = *reinterpret_cast<const float4*>(V + j * 2 * T + 4 * tc);
#pragma unroll
            for (int r = 0; r < RI_MAX; ++r) {
                if (r < RI && i0 + r < N) {
                    const float a = A_res[(i0 + r) * (N + 1) + j];
                    acc[r][0] = fmaf(a, b.x, acc[r][0]);
                    acc[r][1] = fmaf(a, b.y, acc[r][1]);
                    acc[r][2] = fmaf(a, b.z, acc[r][2]);
                    acc[r][3] = fmaf(a, b.w, acc[r][3]);
                }
            }
        }
    } else {
        for (int64_t j0 = 0; j0 < N; j0 += KCH) {
            __syncthreads();   // the previous chunk is consumed
            for (int64_t e = threadIdx.x; e < N * KCH; e += RT) {
                const int64_t i = e / KCH, jj = e - i * KCH;
                stage[i * (KCH + 1) + jj] = (j0 + jj < N) ? __ldg(A_glob + i * N + j0 + jj) : 0.f;
            }
            __syncthreads();
            const int64_t jl = (jmax - j0 < KCH) ? jmax - j0 : KCH;
            for (int64_t jj = 0; jj < jl; ++jj) {
                const float4 b = *reinterpret_cast<const float4*>(V + (j0 + jj) * 2 * T + 4 * tc);
#pragma unroll
                for (int r = 0; r < RI_MAX; ++r) {
                    if (r < RI && i0 + r < N) {
                        const float a = stage[(i0 + r) * (KCH + 1) + jj];
                        acc[r][0] = fmaf(a, b.x, acc[r][0]);
                        acc[r][1] = fmaf(a, b.y, acc[r][1]);
                        acc[r][2] = fmaf(a, b.z, acc[r][2]);
                        acc[r][3] = fmaf(a, b.w, acc[r][3]);
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ int find_prob(const int* start, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int T, bool RES>
__global__ void __launch_bounds__(RT, 1) k_resident(const ResProblem* probs, const int* cta_start, int nprob) {
    constexpr int TC = T / 2, TI = RT / TC;
    extern __shared__ __align__(16) float sm[];
    __shared__ float sS[3 * T], sP[3 * T], sXI[2 * T];
    const int p = find_prob(cta_start, nprob, blockIdx.x);
    const ResProblem& P = probs[p];
    const int64_t N = P.N, M = P.M;
    const int64_t g0 = (int64_t)(blockIdx.x - cta_start[p]) * T;   // first trajectory of this CTA
    float* Sxy = sm;
    float* Sz = Sxy + N * 2 * T;
    float* Pxy = Sz + N * T;
    float* Pz = Pxy + N * 2 * T;
    float* Qxy = Pz + N * T;
    float* mat = Qxy + N * 2 * T;   // W, L (resident) or the chunk buffer
    const int tid = threadIdx.x, tc = tid % TC, ti = tid / TC;
    const int RI = (int)((N + TI - 1) / TI);

    // load the state; trajectories past M get a valid spin and are never stored
    for (int64_t e = tid; e < (int64_t)T * N; e += RT) {
        const int64_t t = e / N, i = e - t * N, m = g0 + t;
        float x = 1.f, y = 1.f, z = -1.f;
        if (m < M) {
            x = P.X[m * N + i];
            y = P.Y[m * N + i];
            z = P.Z[m * N + i];
        }
        Sxy[i * 2 * T + 2 * t] = x;
        Sxy[i * 2 * T + 2 * t + 1] = y;
        Sz[i * T + t] = z;
    }
    if constexpr (RES) {
        float* Ws = mat;
        float* Ls = mat + N * (N + 1);
        for (int64_t e = tid; e < N * N; e += RT) {
            const int64_t i = e / N, j = e - i * N;
            Ws[i * (N + 1) + j] = P.W[e];
            Ls[i * (N + 1) + j] = P.L[e];
        }
    }
    __syncthreads();
    col_sums<T>(Sxy, Sz, N, sS, true);
    __syncthreads();

    const float* Wres = RES ? mat : nullptr;
    const float* Lres = RES ? mat + N * (N + 1) : nullptr;
    float acc[RI_MAX][4];
    unsigned nonfinite = 0;
    for (int64_t k = 0; k < P.steps; ++k) {
        const int64_t ts = P.t0 + k;
        // (a) normals of step ts into P (eta, sites < N) and sXI (xi, site N)
        for (int64_t e = tid; e < (int64_t)T * (N + 1); e += RT) {
            const int64_t i = e / T, t = e - i * T;   // t fastest: consecutive shared-memory columns
            float gx, gy;
            normal2_f32(P.seed, (uint32_t)(P.m0 + g0 + t), (uint32_t)ts, (uint32_t)i, gx, gy);
            if (i < N) {
                Pxy[i * 2 * T + 2 * t] = gx;
                Pxy[i * 2 * T + 2 * t + 1] = gy;
            } else {
                sXI[2 * t] = gx;
                sXI[2 * t + 1] = gy;
            }
        }
        __syncthreads();
        // (b) noise part of the field increment: sqrt(G dt) xi^a - sqrt(dt) (L eta^a)_i
        contract<T, RES, true>(P.L, Lres, mat, Pxy, N, RI, ti, tc, acc);
#pragma unroll
        for (int r = 0; r < RI_MAX; ++r) {
            const int64_t i = (int64_t)ti * RI + r;
            if (r < RI && i < N)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    Qxy[i * 2 * T + 4 * tc + q] = fmaf(-P.sdt, acc[r][q], __fmul_rn(P.sgdt, sXI[4 * tc + q]));
        }
        __syncthreads();   // eta (in P) is consumed, Q is complete
        // (c) W.s and the predictor: Heun s~ = s + s x b(s), or the midpoint state
        contract<T, RES, false>(P.W, Wres, mat, Sxy, N, RI, ti, tc, acc);
#pragma unroll
        for (int r = 0; r < RI_MAX; ++r) {
            const int64_t i = (int64_t)ti * RI + r;
            if (!(r < RI && i < N)) continue;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int t = 2 * tc + u;
                const float x = Sxy[i * 2 * T + 2 * t], y = Sxy[i * 2 * T + 2 * t + 1], z = Sz[i * T + t];
                const float Bxv = fmaf(fmaf(P.G, sS[2 * t], -acc[r][2 * u]), P.hdt, Qxy[i * 2 * T + 2 * t]);
                const float Byv = fmaf(fmaf(P.G, sS[2 * t + 1], -acc[r][2 * u + 1]), P.hdt, Qxy[i * 2 * T + 2 * t + 1]);
                float xp, yp, zp;
                if (P.integ == TWA_INT_MIDPOINT) {
                    mid_rotation_f32(x, y, z, Bxv, Byv, xp, yp, zp);
                } else {
                    xp = __fadd_rn(x, __fmul_rn(z, Bxv));
                    yp = __fadd_rn(y, __fmul_rn(z, Byv));
                    zp = __fadd_rn(z, -fmaf(x, Bxv, __fmul_rn(y, Byv)));
                }
                Pxy[i * 2 * T + 2 * t] = xp;
                Pxy[i * 2 * T + 2 * t + 1] = yp;
                Pz[i * T + t] = zp;
            }
        }
        __syncthreads();
        col_sums<T>(Pxy, Pz, N, sP, false);
        __syncthreads();
        // (d) W.s~ (midpoint: W of the midpoint state) and the corrector
        contract<T, RES, false>(P.W, Wres, mat, Pxy, N, RI, ti, tc, acc);
#pragma unroll
        for (int r = 0; r < RI_MAX; ++r) {
            const int64_t i = (int64_t)ti * RI + r;
            if (!(r < RI && i < N)) continue;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int t = 2 * tc + u;
                const int64_t o = i * 2 * T + 2 * t;
                const float x = Sxy[o], y = Sxy[o + 1], z = Sz[i * T + t];
                const float xp = Pxy[o], yp = Pxy[o + 1], zp = Pz[i * T + t];
                const float Bxv = fmaf(fmaf(P.G, sP[2 * t], -acc[r][2 * u]), P.hdt, Qxy[o]);
                const float Byv = fmaf(fmaf(P.G, sP[2 * t + 1], -acc[r][2 * u + 1]), P.hdt, Qxy[o + 1]);
                float nx, ny, nz;
                if (P.integ == TWA_INT_MIDPOINT) {
                    float mx, my, mz;
                    mid_rotation_f32(x, y, z, Bxv, Byv, mx, my, mz);
                    nx = fmaf(2.0f, mx, -x);
                    ny = fmaf(2.0f, my, -y);
                    nz = fmaf(2.0f, mz, -z);
                } else {
                    // s' = (s + s~)/2 + f(s~)/2
                    const float hx = __fmul_rn(0.5f, __fadd_rn(x, xp));
                    const float hy = __fmul_rn(0.5f, __fadd_rn(y, yp));
                    const float hz = __fmul_rn(0.5f, __fadd_rn(z, zp));
                    nx = fmaf(0.5f, __fmul_rn(zp, Bxv), hx);
                    ny = fmaf(0.5f, __fmul_rn(zp, Byv), hy);
                    nz = fmaf(-0.5f, fmaf(xp, Bxv, __fmul_rn(yp, Byv)), hz);
                }
                if (P.renorm) {
                    const float s = sqrtf(3.0f / fmaf(nx, nx, fmaf(ny, ny, __fmul_rn(nz, nz))));
                    nx = __fmul_rn(nx, s);
                    ny = __fmul_rn(ny, s);
                    nz = __fmul_rn(nz, s);
                }
                if (!(isfinite(nx) && isfinite(ny) && isfinite(nz)) && g0 + t < M) ++nonfinite;
                Sxy[o] = nx;
                Sxy[o + 1] = ny;
                Sz[i * T + t] = nz;
            }
        }
        __syncthreads();
        col_sums<T>(Sxy, Sz, N, sS, true);
        __syncthreads();
        // (e) window moments of the new state, added to the running FP64 sums
        // step by step (the order every route uses, so runs split into several
        // calls give the same bits)
        if (window_sample(ts + 1, P.n_window, P.stride) && tid < T && g0 + tid < M) {
            const double sx = sS[2 * tid], sy = sS[2 * tid + 1], sz = sS[2 * T + tid];
            const double A = 0.25 * (sx * sx + sy * sy);
            double* mm = P.mom + 5 * (g0 + tid);
            mm[0] += sz;
            mm[1] += A;
            mm[2] += A * A;
            mm[3] += A * sz;
            mm[4] += sz * sz;
        }
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)T * N; e += RT) {
        const int64_t t = e / N, i = e - t * N, m = g0 + t;
        if (m < M) {
            P.X[m * N + i] = Sxy[i * 2 * T + 2 * t];
            P.Y[m * N + i] = Sxy[i * 2 * T + 2 * t + 1];
            P.Z[m * N + i] = Sz[i * T + t];
        }
    }
    const unsigned tot = __reduce_add_sync(0xffffffffu, nonfinite);
    if ((tid & 31) == 0 && tot) atomicAdd(&P.flags[FLAG_NONFINITE], (unsigned long long)tot);
}

__global__ void k_f64_to_f32(const double* a, float* b, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) b[e] = (float)a[e];
}

// step counter and window-sample count after a resident launch of `steps` steps
__global__ void k_res_advance(int64_t* d_t, int64_t* d_count, int64_t steps, int64_t samples) {
    *d_t += steps;
    *d_count += samples;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// CTA shape for N sites: the most trajectories per CTA (64, 32, 16, 8) whose
// state fits shared memory next to W and L (resident) or the chunk buffer, and
// whose rows per thread stay within RI_MAX. Returns false if none fits.
bool res_config(int64_t N, int* T, bool* resident, size_t* smem) {
    for (int t : {64, 32, 16, 8}) {
        const int TI = RT / (t / 2);
        if ((N + TI - 1) / TI > RI_MAX) continue;
        for (bool r : {true, false}) {
            const size_t b = sizeof(float) * (res_state_floats(N, t) + res_matrix_floats(N, r));
            if (b <= RES_SMEM_MAX) {
                *T = t;
                *resident = r;
                *smem = b;
                return true;
            }
        }
    }
    return false;
}

int res_prepare(twa_ctx* c) {
    if (c->opts.precision == TWA_PREC_BF16X2) {   // the tensor-core form works on the images of tc
        if (!restc_capable(c))
            return set_error(c, TWA_EUNSUPPORTED, "the tensor-core resident route holds N <= " +
                                                      std::to_string(TWA_RESIDENT_TC_MAX_N) + " sites");
        c->res_tc = true;
        return TWA_OK;
    }
    int T;
    bool r;
    size_t b;
    if (!res_config(c->N, &T, &r, &b))
        return set_error(c, TWA_EUNSUPPORTED, "the resident route holds N <= " + std::to_string(TWA_RESIDENT_MAX_N) +
                                                  " sites");
    const size_t n2 = (size_t)c->N * c->N;
    if (dev_malloc(c, &c->res_W, sizeof(float) * n2) != cudaSuccess ||
        dev_malloc(c, &c->res_L, sizeof(float) * n2) != cudaSuccess)
        return set_error(c, TWA_ENOMEM, "device FP32 copies of W and L");
    k_f64_to_f32<<<nblk((int64_t)n2, 256), 256, 0, c->stream>>>(c->W64, c->res_W, (int64_t)n2);
    k_f64_to_f32<<<nblk((int64_t)n2, 256), 256, 0, c->stream>>>(c->L64, c->res_L, (int64_t)n2);
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

void res_free(twa_ctx* c) {
    dev_free(c, c->res_W);
    dev_free(c, c->res_L);
    c->res_W = c->res_L = nullptr;
}

namespace {
ResProblem problem_of(twa_ctx* c, int64_t steps) {
    ResProblem p{};
    p.W = c->res_W;
    p.L = c->res_L;
    p.X = c->tc->X;
    p.Y = c->tc->Y;
    p.Z = c->tc->Z;
    p.mom = c->mom;
    p.flags = c->d_flags;
    p.M = c->M;
    p.N = c->N;
    p.m0 = c->opts.traj_offset;
    p.t0 = c->steps;
    p.steps = steps;
    p.n_window = c->n_window;
    p.stride = c->n_stride;
    p.seed = c->seed;
    p.G = (float)c->Gamma;
    p.hdt = 0.5f * (float)c->dt;
    p.sgdt = (float)sqrt(c->Gamma * c->dt);
    p.sdt = (float)sqrt(c->dt);
    p.renorm = c->opts.renormalize;
    p.integ = c->opts.integrator;
    return p;
}

int64_t samples_in(const twa_ctx* c, int64_t t0, int64_t steps) {
    int64_t n = 0;
    for (int64_t t = t0 + 1; t <= t0 + steps; ++t) n += window_sample(t, c->n_window, c->n_stride) ? 1 : 0;
    return n;
}

template <int T, bool RES>
int launch_res(twa_ctx* lead, const ResProblem* d_probs, const int* d_start, int nprob, int ctas, size_t smem,
               cudaStream_t st) {
    auto kern = k_resident<T, RES>;
    TWA_CUDA(lead, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RES_SMEM_MAX));
    kern<<<ctas, RT, smem, st>>>(d_probs, d_start, nprob);
    TWA_CUDA(lead, cudaGetLastError());
    return TWA_OK;
}

int launch_shape(twa_ctx* lead, int T, bool r, const ResProblem* d_probs, const int* d_start, int nprob, int ctas,
                 size_t smem, cudaStream_t st) {
#define TWA_RES_CASE(T_, R_) \
    if (T == T_ && r == R_) return launch_res<T_, R_>(lead, d_probs, d_start, nprob, ctas, smem, st);
    TWA_RES_CASE(64, true)
    TWA_RES_CASE(64, false)
    TWA_RES_CASE(32, true)
    TWA_RES_CASE(32, false)
    TWA_RES_CASE(16, true)
    TWA_RES_CASE(16, false)
    TWA_RES_CASE(8, true)
    TWA_RES_CASE(8, false)
#undef TWA_RES_CASE
    return set_error(lead, TWA_EUNSUPPORTED, "resident route: CTA shape not compiled");
}
}  // namespace

// steps[k] steps of every context cs[k] (all on the resident route, trajectories
// fixed), in one launch per CTA shape, on `st`; step counters and sample counts
// advanced. A context with steps[k] = 0 is skipped.
int res_run_many(twa_ctx* const* cs, const int64_t* steps, int n, twa_ctx* lead, cudaStream_t st) {
    // the tensor-core contexts in one launch of their own, the FP32 ones below
    std::vector<int64_t> tc_steps(n, 0), simt_steps(n, 0);
    bool any_tc = false;
    for (int k = 0; k < n; ++k) {
        (cs[k]->res_tc ? tc_steps : simt_steps)[k] = steps[k];
        any_tc = any_tc || (cs[k]->res_tc && steps[k] > 0);
    }
    if (any_tc) {
        const int rc = restc_run_many(cs, tc_steps.data(), n, lead, st);
        if (rc) return rc;
    }
    steps = simt_steps.data();
    struct Item {
        int k, T, ctas;
        bool r;
        size_t smem;
    };
    std::vector<Item> items;
    for (int k = 0; k < n; ++k) {
        if (steps[k] <= 0) continue;
        int T;
        bool r;
        size_t b;
        if (!res_config(cs[k]->N, &T, &r, &b)) return set_error(lead, TWA_EUNSUPPORTED, "resident route: N too large");
        items.push_back({k, T, (int)((cs[k]->M + T - 1) / T), r, b});
    }
    // one launch per CTA shape
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) {
        return a.T != b.T ? a.T > b.T : (int)a.r > (int)b.r;
    });
    size_t i0 = 0;
    while (i0 < items.size()) {
        size_t i1 = i0;
        std::vector<ResProblem> probs;
        std::vector<int> start(1, 0);
        size_t smem = 0;
        while (i1 < items.size() && items[i1].T == items[i0].T && items[i1].r == items[i0].r) {
            probs.push_back(problem_of(cs[items[i1].k], steps[items[i1].k]));
            start.push_back(start.back() + items[i1].ctas);
            smem = std::max(smem, items[i1].smem);
            ++i1;
        }
        const int np = (int)probs.size();
        Scratch<ResProblem> dp(lead, st);
        Scratch<int> ds(lead, st);
        TWA_CUDA(lead, dp.alloc(sizeof(ResProblem) * np));
        TWA_CUDA(lead, ds.alloc(sizeof(int) * (np + 1)));
        TWA_CUDA(lead, cudaMemcpyAsync(dp.p, probs.data(), sizeof(ResProblem) * np, cudaMemcpyHostToDevice, st));
        TWA_CUDA(lead, cudaMemcpyAsync(ds.p, start.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, st));
        // (copies from pageable host memory return once the data is staged, so
        // the host vectors may go out of scope)
        int rc = launch_shape(lead, items[i0].T, items[i0].r, dp.p, ds.p, np, start.back(), smem, st);
        if (rc) return rc;
        i0 = i1;
    }
    for (int k = 0; k < n; ++k) {
        if (steps[k] <= 0) continue;
        twa_ctx* c = cs[k];
        k_res_advance<<<1, 1, 0, st>>>(c->d_t, c->d_count, steps[k], samples_in(c, c->steps, steps[k]));
        TWA_CUDA(lead, cudaGetLastError());
    }
    return TWA_OK;
}

int res_run(twa_ctx* c, int64_t steps) {
    ProfScope p(c, TWA_PROF_RESIDENT);
    twa_ctx* cs[1] = {c};
    return res_run_many(cs, &steps, 1, c, c->stream);
}

}  // namespace twa

// Resident route on the tensor cores (ws_route = TWA_ROUTE_RESIDENT with the
// BF16X2 precision, N <= 128): the BF16X2 step of Eq. S1 -- W and L as BF16
// hi + lo images (of W / w and L / sqrt(w)), the state and the noise rounded
// once to BF16 as operands, FP32 accumulation -- with everything a CTA needs
// resident on its SM for all steps of a call.
//
// One CTA integrates 32 trajectories of one problem (a context, or one point of
// a batched scan). Shared memory holds the four 128 x 128 A images (W hi, W lo,
// L hi, L lo; 128 KB) and three 64 x 128 B images (the state, the predictor and
// the noise eta of the 32 trajectories, rows 2t = x and 2t + 1 = y), all in the
// K-major 128-byte-swizzle layout the MMA reads; TMEM holds two 128 x 64 FP32
// accumulators (L eta, and W s or W s~). Sixteen epilogue warps keep the FP32
// state of their (site, 8 trajectories) in registers across all steps; warp 0
// owns TMEM and issues the MMAs. Per step: the epilogue draws eta (Philox, the
// counters of the dense route) into its image, the MMA warp issues L eta and
// W s, the epilogue forms the noise part and the Heun (or midpoint) predictor
// and writes its image, the MMA warp issues W s~, the epilogue applies the
// corrector, renormalises, writes the new state's image and the collective sums
// (a transpose through shared memory and a fixed-order reduction) and, at window
// steps, the FP64 moments. Generic shared-memory stores feed the MMAs through
// fence.proxy.async; MMA completion is an mbarrier with a bounded wait.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "twa_internal.cuh"

namespace twa {
namespace {

constexpr int RC_T = 32;                        // trajectories per CTA
constexpr int RC_NB = 2 * RC_T;                 // B rows = MMA N: x and y of each trajectory
constexpr int RC_WARPS = 16;                    // four per TMEM lane quadrant; warp 0 also issues the MMAs
constexpr int RC_THREADS = 32 * RC_WARPS;
constexpr int RC_A_CHUNK = 128 * 128;           // bytes of a 128-row x 64-K BF16 tile
constexpr int RC_B_CHUNK = RC_NB * 128;         // a 64-row x 64-K tile
constexpr int RC_A_IMG = 2 * RC_A_CHUNK;        // K = 128
constexpr int RC_B_IMG = 2 * RC_B_CHUNK;
constexpr int RC_OFF_B = 4 * RC_A_IMG;          // A images: W hi, W lo, L hi, L lo
constexpr int RC_OFF_SMALL = RC_OFF_B + 3 * RC_B_IMG;   // B images: state, predictor, eta
constexpr int RC_SMEM = RC_OFF_SMALL + 8192 + 1024;     // small arrays, 1024-byte alignment slack
constexpr unsigned long long RC_WAIT_NS = 2000000000ull;
// instruction descriptor: D F32, A and B BF16, both K-major, N = 64, M = 128
constexpr uint32_t RC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(RC_NB >> 3) << 17) | ((128u >> 4) << 24);

struct RcProblem {
    const __nv_bfloat16 *Whi, *Wlo, *Lhi, *Llo;   // [N][ldk] images of W / w and L / sqrt(w)
    float *X, *Y, *Z;                             // state [M][N]
    double* mom;                                  // window sums [M][5]
    unsigned long long* flags;
    int64_t M, N, ldk, m0, t0, steps, n_window, stride;
    uint64_t seed;
    float hdtG, hdtw, sgdt, sdt;                  // dt G / 2, dt w / 2, sqrt(G dt), sqrt(w dt)
    int renorm, integ;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of BF16 element (row, k) in a K-major tile of 64-wide K chunks
// (`chunk` bytes each) with the 128-byte swizzle: 16-byte piece c of a 128-byte
// row r sits at piece c ^ (r mod 8)
__device__ __forceinline__ uint32_t swz(int row, int k, int chunk) {
    const int kc = k >> 6, kk = k & 63;
    return (uint32_t)(kc * chunk + row * 128 + ((((kk >> 3) ^ (row & 7)) << 4) | ((kk & 7) << 1)));
}

// shared-memory descriptor of such a tile: 8-row atoms 1024 bytes apart,
// descriptor version 1, layout code 2 (128-byte swizzle)
__device__ __forceinline__ uint64_t rc_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void rc_mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtm),
        "l"(ad), "l"(bd), "r"(RC_IDESC), "r"(acc));
}

__device__ __forceinline__ void rc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// D (+)= A_h B over the K chunks holding nonzero entries, for h = 0, 1 (the hi
// and lo images at a, a + RC_A_IMG); `acc0` = 0 starts the sum afresh
__device__ __forceinline__ void rc_mma_pair(uint32_t dtm, uint32_t a, uint32_t b, int nkc, uint32_t acc0) {
    for (int h = 0; h < 2; ++h)
        for (int kc = 0; kc < nkc; ++kc)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                rc_mma(dtm, rc_desc(a + h * RC_A_IMG + kc * RC_A_CHUNK + kk * 32), rc_desc(b + kc * RC_B_CHUNK + kk * 32),
                       (acc0 | h | kc | kk) ? 1u : 0u);
}

__device__ __forceinline__ bool rc_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase of the given parity; a timeout is counted in
// flags[FLAG_TIMEOUT]
__device__ __noinline__ bool rc_wait(uint64_t* bar, uint32_t parity, unsigned long long* flags) {
    if (rc_try(bar, parity)) return true;
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (true) {
        if (rc_try(bar, parity)) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > RC_WAIT_NS) {
            atomicAdd(&flags[FLAG_TIMEOUT], 1ull);
            return false;
        }
    }
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor core's reads
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 16 consecutive FP32 accumulator columns
__device__ __forceinline__ void rc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

// Sums over the warp's 32 lanes of NV values (NV a power of two <= 32) by
// recursive halving: at each of log2(NV) exchange rounds a lane keeps the half
// of its live values selected by one bit of its lane index and adds its
// partner's copy of that half; the remaining rounds are a plain butterfly. On
// return every lane holds the sum of value index lane / (32 / NV), the same bits
// on all 32 / NV lanes that hold it; the order of the additions is fixed.
template <int NV>
__device__ __forceinline__ float warp_sum_scatter(float (&v)[NV], int lane) {
#pragma unroll
    for (int h = NV / 2, off = 16; h >= 1; h >>= 1, off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float send = up ? v[k] : v[k + h];
            const float keep = up ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    float s = v[0];
#pragma unroll
    for (int off = 16 / NV; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}

// Sum of the four lane quadrants' partial sums of column c, in quadrant order.
__device__ __forceinline__ float quad_sum(const float* part, int stride, int c) {
    return __fadd_rn(__fadd_rn(__fadd_rn(part[c], part[stride + c]), part[2 * stride + c]), part[3 * stride + c]);
}

__global__ void __launch_bounds__(RC_THREADS, 1) k_restc(const RcProblem* probs, const int* cta_start, int nprob) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    int p = 0;
    while (p + 1 < nprob && cta_start[p + 1] <= (int)blockIdx.x) ++p;
    const RcProblem& P = probs[p];
    const int64_t mbase = (int64_t)((int)blockIdx.x - cta_start[p]) * RC_T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, e = threadIdx.x;
    uint8_t* A = sm;
    uint8_t* Bs = sm + RC_OFF_B;     // image of the state
    uint8_t* Bp = Bs + RC_B_IMG;     // of the predictor (midpoint scheme: of the midpoint state)
    uint8_t* Be = Bp + RC_B_IMG;     // of eta
    float* S = (float*)(sm + RC_OFF_SMALL);   // [64] sums over sites of x, y of the state (column 2t, 2t + 1)
    float* Sp = S + RC_NB;                     // [64] ... of the predictor
    float* XI = Sp + RC_NB;                    // [64] collective normals
    float* part = XI + RC_NB;                  // [4][64] per lane quadrant partial sums of x, y
    float* partz = part + 4 * RC_NB;           // [4][32] ... of z
    uint64_t* bar = (uint64_t*)(partz + 4 * RC_T);
    uint32_t* tslot = (uint32_t*)(bar + 2);
    double* mom = (double*)(tslot + 2);        // [32][5]

    const int N = (int)P.N;
    const int nkc = (N + 63) >> 6;             // 64-wide K chunks with nonzero entries

    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar[0])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // W hi, W lo, L hi, L lo into the swizzled A tiles (zero beyond N)
    for (int u = threadIdx.x; u < 4 * 2048; u += RC_THREADS) {
        const int im = u >> 11, rem = u & 2047, kc = rem >> 10, row = (rem >> 3) & 127, c = rem & 7;
        const int col = kc * 64 + c * 8;
        const __nv_bfloat16* img = im == 0 ? P.Whi : im == 1 ? P.Wlo : im == 2 ? P.Lhi : P.Llo;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < N && col < P.ldk) v = *(const uint4*)(img + (int64_t)row * P.ldk + col);
        *(uint4*)(A + im * RC_A_IMG + kc * RC_A_CHUNK + row * 128 + ((c ^ (row & 7)) << 4)) = v;
    }
    // the running window sums of the CTA's trajectories (continued in the same
    // order as one longer call would add them)
    for (int k = threadIdx.x; k < RC_T * 5; k += RC_THREADS) {
        const int64_t m = mbase + k / 5;
        mom[k] = m < P.M ? P.mom[m * 5 + k % 5] : 0.0;
    }

    // thread (warp, lane): TMEM lane quadrant q = warp mod 4 (the lanes a warp
    // may read), site i = 32 q + lane, trajectories 8 g .. 8 g + 7 (accumulator
    // columns 16 g .. 16 g + 15), g = warp / 4
    const int q = warp & 3, g = warp >> 2, i = 32 * q + lane;
    const bool site_ok = i < N;
    float x[8], y[8], z[8];
    bool traj_ok[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        x[j] = y[j] = z[j] = 0.f;
        const int64_t m = mbase + 8 * g + j;
        traj_ok[j] = site_ok && m < P.M;
        if (traj_ok[j]) {
            const int64_t o = m * N + i;
            x[j] = P.X[o];
            y[j] = P.Y[o];
            z[j] = P.Z[o];
        }
    }
    // BF16 image of (vx, vy) and the quadrant's partial sums over its sites
    auto put_state = [&](uint8_t* Bimg, const float* vx, const float* vy) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = 2 * (8 * g + j);
            *(__nv_bfloat16*)(Bimg + swz(n, i, RC_B_CHUNK)) = __float2bfloat16_rn(vx[j]);
            *(__nv_bfloat16*)(Bimg + swz(n + 1, i, RC_B_CHUNK)) = __float2bfloat16_rn(vy[j]);
            v[2 * j] = vx[j];
            v[2 * j + 1] = vy[j];
        }
        const float s = warp_sum_scatter<16>(v, lane);
        if (!(lane & 1)) part[q * RC_NB + 16 * g + (lane >> 1)] = s;
    };
    // eta of step t into its image (zero rows beyond N) and the collective
    // normals xi of step t (counter i = N); warp w draws xi of trajectories 2w, 2w + 1
    auto draw_noise = [&](int64_t t) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int tl = 8 * g + j;
            float gx = 0.f, gy = 0.f;
            if (site_ok) normal2_f32(P.seed, (uint32_t)(P.m0 + mbase + tl), (uint32_t)t, (uint32_t)i, gx, gy);
            *(__nv_bfloat16*)(Be + swz(2 * tl, i, RC_B_CHUNK)) = __float2bfloat16_rn(gx);
            *(__nv_bfloat16*)(Be + swz(2 * tl + 1, i, RC_B_CHUNK)) = __float2bfloat16_rn(gy);
        }
        if (lane < 2) {
            const int tl = 2 * warp + lane;
            float gx, gy;
            normal2_f32(P.seed, (uint32_t)(P.m0 + mbase + tl), (uint32_t)t, (uint32_t)N, gx, gy);
            XI[2 * tl] = gx;
            XI[2 * tl + 1] = gy;
        }
    };

    if (P.steps > 0) draw_noise(P.t0);
    put_state(Bs, x, y);
    proxy_fence();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot, accL = tmem, accW = tmem + RC_NB;
    if (e < RC_NB) S[e] = quad_sum(part, RC_NB, e);
    __syncthreads();

    const uint32_t trow = ((uint32_t)(32 * q) << 16);   // this warp's lane quadrant in TMEM addresses
    const float hdtG = P.hdtG, hdtw = P.hdtw, sgdt = P.sgdt, sdt = P.sdt;
    uint32_t phase = 0;
    unsigned bad = 0;
    bool ok = true;
    for (int64_t s = 0; s < P.steps && ok; ++s) {
        const int64_t t = P.t0 + s;
        // ---- L eta and W s (eta, the state's image and S are in place) ----
        if (e == 0) {
            tc_after();
            rc_mma_pair(accL, smem_u32(A + 2 * RC_A_IMG), smem_u32(Be), nkc, 0u);
            rc_mma_pair(accW, smem_u32(A), smem_u32(Bs), nkc, 0u);
            rc_commit(&bar[0]);
        }
        // ---- noise part and predictor ----
        float bnx[8], bny[8], xp[8], yp[8], zp[8];
        bool w_ok = rc_wait(&bar[0], phase, P.flags);
        tc_after();
        {
            float qv[16], pv[16];
            rc_ld16(accL + trow + 16 * g, qv);
            rc_ld16(accW + trow + 16 * g, pv);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int tl = 8 * g + j;
                // sqrt(G dt) xi - sqrt(w dt) (L1 eta); B = 1/2 (G S - w P1) dt + noise part
                bnx[j] = fmaf(-sdt, qv[2 * j], __fmul_rn(sgdt, XI[2 * tl]));
                bny[j] = fmaf(-sdt, qv[2 * j + 1], __fmul_rn(sgdt, XI[2 * tl + 1]));
                const float Bx = fmaf(-hdtw, pv[2 * j], fmaf(hdtG, S[2 * tl], bnx[j]));
                const float By = fmaf(-hdtw, pv[2 * j + 1], fmaf(hdtG, S[2 * tl + 1], bny[j]));
                if (P.integ == TWA_INT_MIDPOINT) {
                    mid_rotation_f32(x[j], y[j], z[j], Bx, By, xp[j], yp[j], zp[j]);
                } else {
                    xp[j] = __fadd_rn(x[j], __fmul_rn(z[j], Bx));
                    yp[j] = __fadd_rn(y[j], __fmul_rn(z[j], By));
                    zp[j] = __fadd_rn(z[j], -fmaf(x[j], Bx, __fmul_rn(y[j], By)));
                }
                if (!traj_ok[j]) xp[j] = yp[j] = zp[j] = 0.f;
            }
        }
        put_state(Bp, xp, yp);
        proxy_fence();
        tc_before();
        ok = !__syncthreads_or(!w_ok);
        phase ^= 1u;
        if (!ok) break;
        // ---- W s~ (the accumulator has been read); meanwhile Sp and the
        // noise of the next step (L eta has been read too) ----
        if (e == 0) {
            tc_after();
            rc_mma_pair(accW, smem_u32(A), smem_u32(Bp), nkc, 0u);
            rc_commit(&bar[0]);
        }
        if (e < RC_NB) Sp[e] = quad_sum(part, RC_NB, e);
        if (s + 1 < P.steps) draw_noise(t + 1);
        proxy_fence();
        __syncthreads();
        // ---- corrector, renormalisation, the new state's image and sums ----
        w_ok = rc_wait(&bar[0], phase, P.flags);
        tc_after();
        {
            float pv[16];
            rc_ld16(accW + trow + 16 * g, pv);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int tl = 8 * g + j;
                const float Bx = fmaf(-hdtw, pv[2 * j], fmaf(hdtG, Sp[2 * tl], bnx[j]));
                const float By = fmaf(-hdtw, pv[2 * j + 1], fmaf(hdtG, Sp[2 * tl + 1], bny[j]));
                float nx, ny, nz;
                if (P.integ == TWA_INT_MIDPOINT) {
                    // s' = 2 m - s of the rotation of s by the midpoint state's field
                    float mx, my, mz;
                    mid_rotation_f32(x[j], y[j], z[j], Bx, By, mx, my, mz);
                    nx = fmaf(2.0f, mx, -x[j]);
                    ny = fmaf(2.0f, my, -y[j]);
                    nz = fmaf(2.0f, mz, -z[j]);
                } else {
                    // s' = (s + s~)/2 + f(s~)/2
                    const float hx = __fmul_rn(0.5f, __fadd_rn(x[j], xp[j]));
                    const float hy = __fmul_rn(0.5f, __fadd_rn(y[j], yp[j]));
                    const float hz = __fmul_rn(0.5f, __fadd_rn(z[j], zp[j]));
                    nx = fmaf(0.5f, __fmul_rn(zp[j], Bx), hx);
                    ny = fmaf(0.5f, __fmul_rn(zp[j], By), hy);
                    nz = fmaf(-0.5f, fmaf(xp[j], Bx, __fmul_rn(yp[j], By)), hz);
                }
                if (P.renorm) {
                    const float r = sqrtf(3.0f / fmaf(nx, nx, fmaf(ny, ny, __fmul_rn(nz, nz))));
                    nx = __fmul_rn(nx, r);
                    ny = __fmul_rn(ny, r);
                    nz = __fmul_rn(nz, r);
                }
                if (traj_ok[j]) {
                    if (!(isfinite(nx) && isfinite(ny) && isfinite(nz))) ++bad;
                    x[j] = nx;
                    y[j] = ny;
                    z[j] = nz;
                }
            }
        }
        put_state(Bs, x, y);
        const bool sample = window_sample(t + 1, P.n_window, P.stride);
        if (sample) {   // partial sums of S^z
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = z[j];
            const float sz = warp_sum_scatter<8>(v, lane);
            if (!(lane & 3)) partz[q * RC_T + 8 * g + (lane >> 2)] = sz;
        }
        proxy_fence();
        tc_before();
        ok = !__syncthreads_or(!w_ok);
        phase ^= 1u;
        if (!ok) break;
        // ---- S of the new state; at window steps the FP64 moments ----
        if (e < RC_T) {
            const float sx = quad_sum(part, RC_NB, 2 * e), sy = quad_sum(part, RC_NB, 2 * e + 1);
            S[2 * e] = sx;
            S[2 * e + 1] = sy;
            if (sample) {
                const double dx = sx, dy = sy, sz = quad_sum(partz, RC_T, e);
                const double Av = 0.25 * (dx * dx + dy * dy);
                double* mm = mom + 5 * e;
                mm[0] += sz;
                mm[1] += Av;
                mm[2] += Av * Av;
                mm[3] += Av * sz;
                mm[4] += sz * sz;
            }
        }
        __syncthreads();
    }
    // after a timed-out wait, the MMAs of the abandoned step finish before TMEM
    // is freed (a bounded wait on the commit it would have waited for)
    if (!ok && e == 0) rc_wait(&bar[0], phase ^ 1u, P.flags);
    // state and window sums back to global memory
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (traj_ok[j]) {
            const int64_t o = (mbase + 8 * g + j) * N + i;
            P.X[o] = x[j];
            P.Y[o] = y[j];
            P.Z[o] = z[j];
        }
    }
    const unsigned nb = __reduce_add_sync(0xffffffffu, bad);
    if (lane == 0 && nb) atomicAdd(&P.flags[FLAG_NONFINITE], (unsigned long long)nb);
    if (e < RC_T && mbase + e < P.M)
        for (int k = 0; k < 5; ++k) P.mom[(mbase + e) * 5 + k] = mom[5 * e + k];
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
    }
}

__global__ void k_rc_advance(int64_t* d_t, int64_t* d_count, int64_t steps, int64_t samples) {
    *d_t += steps;
    *d_count += samples;
}

RcProblem problem_of(twa_ctx* c, int64_t steps) {
    const TcState* t = c->tc;
    RcProblem p{};
    p.Whi = t->Whi;
    p.Wlo = t->Wlo;
    p.Lhi = t->Lhi;
    p.Llo = t->Llo;
    p.X = t->X;
    p.Y = t->Y;
    p.Z = t->Z;
    p.mom = c->mom;
    p.flags = c->d_flags;
    p.M = c->M;
    p.N = c->N;
    p.ldk = t->ldk;
    p.m0 = c->opts.traj_offset;
    p.t0 = c->steps;
    p.steps = steps;
    p.n_window = c->n_window;
    p.stride = c->n_stride;
    p.seed = c->seed;
    // the images hold W / w and L / sqrt(w): the factors of the dense route's epilogue
    p.hdtG = (float)(0.5 * c->dt * c->Gamma);
    p.hdtw = (float)(0.5 * c->dt * t->wsc);
    p.sgdt = (float)sqrt(c->Gamma * c->dt);
    p.sdt = (float)(sqrt(c->dt) * t->lsc);
    p.renorm = c->opts.renormalize;
    p.integ = c->opts.integrator;
    return p;
}

int64_t samples_in(const twa_ctx* c, int64_t t0, int64_t steps) {
    int64_t n = 0;
    for (int64_t t = t0 + 1; t <= t0 + steps; ++t) n += window_sample(t, c->n_window, c->n_stride) ? 1 : 0;
    return n;
}

}  // namespace

bool restc_capable(const twa_ctx* c) { return c->opts.precision == TWA_PREC_BF16X2 && c->N <= TWA_RESIDENT_TC_MAX_N; }

// steps[k] steps of every context cs[k] (resident route, BF16X2, N <= 128) in one
// launch, on `st`; step counters and sample counts advanced. Contexts with
// steps[k] = 0 are skipped.
int restc_run_many(twa_ctx* const* cs, const int64_t* steps, int n, twa_ctx* lead, cudaStream_t st) {
    std::vector<RcProblem> probs;
    std::vector<int> start(1, 0);
    for (int k = 0; k < n; ++k) {
        if (steps[k] <= 0) continue;
        if (!restc_capable(cs[k]))
            return set_error(lead, TWA_EUNSUPPORTED, "tensor-core resident route: BF16X2 and N <= 128");
        probs.push_back(problem_of(cs[k], steps[k]));
        start.push_back(start.back() + (int)((cs[k]->M + RC_T - 1) / RC_T));
    }
    if (!probs.empty()) {
        const int np = (int)probs.size();
        Scratch<RcProblem> dp(lead, st);
        Scratch<int> ds(lead, st);
        TWA_CUDA(lead, dp.alloc(sizeof(RcProblem) * np));
        TWA_CUDA(lead, ds.alloc(sizeof(int) * (np + 1)));
        TWA_CUDA(lead, cudaMemcpyAsync(dp.p, probs.data(), sizeof(RcProblem) * np, cudaMemcpyHostToDevice, st));
        TWA_CUDA(lead, cudaMemcpyAsync(ds.p, start.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, st));
        TWA_CUDA(lead, cudaFuncSetAttribute(k_restc, cudaFuncAttributeMaxDynamicSharedMemorySize, RC_SMEM));
        k_restc<<<start.back(), RC_THREADS, RC_SMEM, st>>>(dp.p, ds.p, np);
        TWA_CUDA(lead, cudaGetLastError());
    }
    for (int k = 0; k < n; ++k) {
        if (steps[k] <= 0) continue;
        twa_ctx* c = cs[k];
        k_rc_advance<<<1, 1, 0, st>>>(c->d_t, c->d_count, steps[k], samples_in(c, c->steps, steps[k]));
        TWA_CUDA(lead, cudaGetLastError());
    }
    return TWA_OK;
}

}  // namespace twa

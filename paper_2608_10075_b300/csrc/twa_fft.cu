// Toeplitz route for the pump field of Eq. S1. The pump matrix of Eq. 2 depends
// only on |i - j|, so sum_j w_ij s_j is a linear convolution of s with
// c_d = w / (1 + d)^alpha. On a circle of even length P >= 2N - 2 the sequence
// c_{min(d, P-d)}, d < P, is the first column of a symmetric circulant C whose
// leading N x N block is W (every |i - j| < N is at most P / 2), so
// W s = first N entries of IFFT(lambda . FFT(s, zero padded)), lambda = FFT of
// that column (real, because the column is symmetric). The sequence is convex
// and decreasing on 0..P/2, so lambda >= 0 (Dietrich-Newsam) and the same C
// also draws the pump noise: with Z_k complex standard normal (Philox stream 2),
// Y = IFFT-direction sum of sqrt(lambda_k / P) Z_k has Re Y and Im Y independent
// with covariance C, i.e. chi^x and chi^y with covariance W on the first N sites.
//
// Since W is real, one complex transform of z = s^x + i s^y gives both
// components: W z = W s^x + i W s^y. One CTA holds one trajectory's transform in
// shared memory (P complex FP32 values, P = 2^a 3^b 5^c <= 28000), runs an
// in-place mixed-radix decimation-in-frequency FFT whose output is in digit-
// reversed order, multiplies by lambda stored in that same order, and runs the
// inverse as decimation in time, which takes digit-reversed input and returns
// natural order: no permutation pass. The Heun predictor / corrector of the
// trajectory then run in the same kernel, with the collective sums S^a reduced
// in the block.
//
// Longer transforms (P > 28000, N > 14001) spread one trajectory over a cluster
// of C = 2, 4 or 8 CTAs on as many SMs: position p lives in the shared memory of
// CTA p mod C at offset p / C. A butterfly of stride m touches positions
// congruent mod C when C divides m, so with the radices ordered 5s, 3s, 2s, 4s
// (the strides of all stages but the last are then multiples of 4 C or more)
// every stage is local to one CTA except the middle one (stride 1), which reads
// and writes the other CTAs' shared memory (distributed shared memory,
// ld/st.shared::cluster) between two cluster barriers.
#include <math.h>
#include <stdlib.h>

#include <type_traits>

#include "twa_internal.cuh"

namespace twa {
namespace {

constexpr int FT = 1024;                 // threads per CTA
constexpr int64_t FFT_MAX_PLOC = 28000;  // complex FP32 values of one CTA's share of the transform (219 KB)
constexpr int FFT_MAX_C = 8;             // CTAs per trajectory (portable cluster size)
// two-level twiddles: w^n = hi[n / LO] lo[n % LO]; LO = 128 for one CTA (hi table
// <= 219 entries at P <= 28000), 256 for clusters (P <= 120000 at N <= 60000)
template <int C>
struct TwCfg {
    static constexpr int LOG = C == 1 ? 7 : 8;
    static constexpr int LO = 1 << LOG;
    // lo entry k is stored at k + k / 16: the strided lookups n = j * step of the
    // middle stages (step a multiple of 16 or 32) then fall on distinct banks
    static constexpr int PADDED = LO + LO / 16;
};
__host__ __device__ constexpr int lo_slot(int k) { return k + (k >> 4); }
template <int C>
__host__ __device__ constexpr int log2c() { return C == 1 ? 0 : C == 2 ? 1 : C == 4 ? 2 : 3; }

struct FftArgs {
    int64_t N, M, P;
    int nst;
    int radix[40];
    unsigned local_mask;                 // bit s: stage s (stride m_s) stays inside one CTA of the cluster
    int wl;                              // one CTA: stages s >= wl run warp by warp (nst: none)
    int Lw;                              // span of stage wl's blocks: each warp owns whole blocks
    const float2* dtw;                   // one CTA: direct twiddle tables of the stages that have one
    int dtw_off[40];                     // offset of stage s's table in dtw (-1: two-level lookup)
    int dtw_total;                       // entries of all direct tables
    const float* lam;
    const float2* tw;
    float G, dt;
    int renorm;
    int integ;                           // TWA_INT_HEUN or TWA_INT_MIDPOINT
    const float *X, *Y, *Z;              // PRED: s; CORR: s~ (midpoint scheme: the midpoint state)
    const float *X0, *Y0, *Z0;           // CORR: s, the state before the step
    const float *Bnx, *Bny;              // noise part of the field increment
    float *oX, *oY, *oZ;                 // PRED: s~ (midpoint scheme: (s + s~)/2); CORR: s'
    double* mom;                         // CORR: window sums [M][5]
    int64_t* d_t;
    int64_t* d_count;
    int64_t n_window, n_stride;
    unsigned long long* flags;
    const double* field_in;              // FIELD: [K][N]
    double* field_out;
    int64_t K;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// ---------------------------------------------------------------------------
// cluster helpers: rank, barrier, distributed shared memory
template <int C>
__device__ __forceinline__ int cl_rank() {
    if constexpr (C == 1) return 0;
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// barrier between two stages: the cluster's when either reads or writes another
// CTA's shared memory, the block's otherwise
template <int C>
__device__ __forceinline__ void stage_sync(bool cluster) {
    if constexpr (C > 1) {
        if (cluster) {
            cl_sync();
            return;
        }
    }
    __syncthreads();
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 cl_ld(uint32_t a) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void cl_st(uint32_t a, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ float cl_ldf(uint32_t a) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}

// Radix-R DFT in registers: y_k = sum_q a_q exp(-+ 2 pi i q k / R) (INV: +).
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* a) {
    if (R == 2) {
        const float2 t = a[1];
        a[1] = csub(a[0], t);
        a[0] = cadd(a[0], t);
    } else if (R == 4) {
        const float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        const float2 t2 = cadd(a[1], a[3]), t3 = csub(a[1], a[3]);
        // forward: y1 = t1 - i t3, y3 = t1 + i t3; inverse: the signs swap
        const float2 mi = INV ? make_float2(-t3.y, t3.x) : make_float2(t3.y, -t3.x);
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, mi);
        a[3] = csub(t1, mi);
    } else if (R == 3) {
        const float h = 0.86602540378443865f;   // sin(2 pi / 3)
        const float2 s = cadd(a[1], a[2]), d = csub(a[1], a[2]);
        const float2 m = make_float2(a[0].x - 0.5f * s.x, a[0].y - 0.5f * s.y);
        // forward: y1 = m - i h d, y2 = m + i h d
        const float2 ihd = INV ? make_float2(-h * d.y, h * d.x) : make_float2(h * d.y, -h * d.x);
        a[0] = cadd(a[0], s);
        a[1] = cadd(m, ihd);
        a[2] = csub(m, ihd);
    } else {   // R == 5
        const float c1 = 0.30901699437494742f, s1 = 0.95105651629515357f;   // cos, sin of 2 pi / 5
        const float c2 = -0.80901699437494742f, s2 = 0.58778525229247313f;  // cos, sin of 4 pi / 5
        const float2 p1 = cadd(a[1], a[4]), m1 = csub(a[1], a[4]);
        const float2 p2 = cadd(a[2], a[3]), m2 = csub(a[2], a[3]);
        const float2 r1 = make_float2(a[0].x + c1 * p1.x + c2 * p2.x, a[0].y + c1 * p1.y + c2 * p2.y);
        const float2 r2 = make_float2(a[0].x + c2 * p1.x + c1 * p2.x, a[0].y + c2 * p1.y + c1 * p2.y);
        // imaginary parts: sum of sin terms times (a_q - a_{5-q})
        const float2 q1 = make_float2(s1 * m1.x + s2 * m2.x, s1 * m1.y + s2 * m2.y);
        const float2 q2 = make_float2(s2 * m1.x - s1 * m2.x, s2 * m1.y - s1 * m2.y);
        // forward: y1 = r1 - i q1, y4 = r1 + i q1, y2 = r2 - i q2, y3 = r2 + i q2
        const float2 iq1 = INV ? make_float2(-q1.y, q1.x) : make_float2(q1.y, -q1.x);
        const float2 iq2 = INV ? make_float2(-q2.y, q2.x) : make_float2(q2.y, -q2.x);
        a[0] = cadd(a[0], cadd(p1, p2));
        a[1] = cadd(r1, iq1);
        a[4] = csub(r1, iq1);
        a[2] = cadd(r2, iq2);
        a[3] = csub(r2, iq2);
    }
}

// Twiddles w^n = exp(-2 pi i n / P) from two small shared-memory tables:
// w^n = hi[n / LO] * lo[n % LO] (one complex product, FP32 accurate).
template <int C>
struct Tw {
    const float2* hi;
    const float2* lo;
    __device__ __forceinline__ float2 operator[](int n) const {
        return cmul(hi[n >> TwCfg<C>::LOG], lo[lo_slot(n & (TwCfg<C>::LO - 1))]);
    }
};

// One stage over butterflies of radix R and stride m (span L = m R): DIF applies
// the small DFT then the twiddles w_L^{jk}; DIT (inverse) undoes the twiddles,
// then the inverse DFT. w_L^{jk} = w^{j k P / L} = (w^{j P / L})^k: one table
// lookup per butterfly, the higher powers by complex products (k < R <= 5).
// The butterfly's R inputs come from `ld(position)` and its outputs go to
// `st(position, value)`: shared memory inside the transform, global memory in
// the first and last stages, which thereby replace separate load/store passes.
// CTA `rank` of a cluster of C runs the butterflies u = rank (mod C): when C
// divides m, all R positions of such a butterfly are = rank (mod C), i.e. in its
// own shared memory.
template <int R, bool INV, int C, typename LD, typename ST>
__device__ __forceinline__ void stage_io(int P, int m, const Tw<C> tw, LD& ld, ST& st, int rank,
                                         const float2* ds) {
    const int L = m * R, step = P / L, nb = P / R;   // P <= 120000: 32-bit indices
    constexpr int U = FT * C;
    // butterfly u = b m + j; advancing u by U advances (b, j) by (db, dj), with
    // one carry: no integer division inside the loop
    const int db = U / m, dj = U - db * m;
    const int u0 = rank + C * (int)threadIdx.x;
    int b = u0 / m, j = u0 - b * m;
    for (int u = u0; u < nb; u += U) {
        const int jc = j, base = b * L + j;
        b += db;
        j += dj;
        if (j >= m) {
            j -= m;
            ++b;
        }
        float2 a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = ld(base + q * m);
        float2 w[R];
        // w_L^j: this stage's direct table (one load), or the two-level lookup
        w[1] = ds ? ds[jc] : tw[jc * step];
#pragma unroll
        for (int k = 2; k < R; ++k) w[k] = cmul(w[k - 1], w[1]);
        if (!INV) {
            dft<R, false>(a);
#pragma unroll
            for (int k = 1; k < R; ++k) a[k] = cmul(a[k], w[k]);
        } else {
#pragma unroll
            for (int k = 1; k < R; ++k) a[k] = cmulc(a[k], w[k]);
            dft<R, true>(a);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) st(base + q * m, a[q]);
    }
}

template <bool INV, int C, typename LD, typename ST>
__device__ __forceinline__ void stage_any(int r, int P, int m, const Tw<C> tw, LD& ld, ST& st, int rank,
                                          const float2* ds = nullptr) {
    switch (r) {
        case 4: stage_io<4, INV, C>(P, m, tw, ld, st, rank, ds); break;
        case 2: stage_io<2, INV, C>(P, m, tw, ld, st, rank, ds); break;
        case 3: stage_io<3, INV, C>(P, m, tw, ld, st, rank, ds); break;
        default: stage_io<5, INV, C>(P, m, tw, ld, st, rank, ds); break;
    }
}

// Last forward stage, product with the spectrum and first inverse stage in one
// pass: all three work on the same groups of R neighbouring positions (stride
// m = 1, twiddles 1), so each group stays in registers.
template <int R, int C, typename LD, typename ST>
__device__ __forceinline__ void middle_io(int P, const float* __restrict__ lam, LD& ld, ST& st, int rank) {
    for (int u = rank + C * (int)threadIdx.x; u < P / R; u += FT * C) {
        const int base = u * R;
        float2 a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = ld(base + q);
        dft<R, false>(a);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const float l = __ldg(&lam[base + q]);
            a[q] = make_float2(a[q].x * l, a[q].y * l);
        }
        dft<R, true>(a);
#pragma unroll
        for (int q = 0; q < R; ++q) st(base + q, a[q]);
    }
}

template <int C, typename LD, typename ST>
__device__ __forceinline__ void middle_any(int r, int P, const float* lam, LD& ld, ST& st, int rank) {
    switch (r) {
        case 4: middle_io<4, C>(P, lam, ld, st, rank); break;
        case 2: middle_io<2, C>(P, lam, ld, st, rank); break;
        case 3: middle_io<3, C>(P, lam, ld, st, rank); break;
        default: middle_io<5, C>(P, lam, ld, st, rank); break;
    }
}

// The same stage with the butterflies of whole blocks of span Lw (a block of
// stage wl: it holds entire blocks of every later stage) given to one warp each:
// warp w takes blocks w, w + 32, ...; within a block, butterfly t = b' m + j
// (sub-block b' of span L = m R, offset j) goes to lane t mod 32. Consecutive
// warp-local stages then touch only the warp's own positions and need a warp
// barrier instead of a block barrier. Same butterflies, same arithmetic.
template <int R, bool INV, typename LD, typename ST>
__device__ __forceinline__ void stage_warp(int P, int m, int Lw, const Tw<1> tw, LD& ld, ST& st, const float2* ds) {
    const int L = m * R, step = P / L, per = Lw / R, ntop = P / Lw;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int db = 32 / m, dj = 32 - db * m;
    for (int B = warp; B < ntop; B += FT / 32) {
        const int top = B * Lw;
        int b = lane / m, j = lane - b * m;
        for (int t = lane; t < per; t += 32) {
            const int jc = j, base = top + b * L + j;
            b += db;
            j += dj;
            if (j >= m) {
                j -= m;
                ++b;
            }
            float2 a[R];
#pragma unroll
            for (int q = 0; q < R; ++q) a[q] = ld(base + q * m);
            float2 w[R];
            w[1] = ds ? ds[jc] : tw[jc * step];
#pragma unroll
            for (int k = 2; k < R; ++k) w[k] = cmul(w[k - 1], w[1]);
            if (!INV) {
                dft<R, false>(a);
#pragma unroll
                for (int k = 1; k < R; ++k) a[k] = cmul(a[k], w[k]);
            } else {
#pragma unroll
                for (int k = 1; k < R; ++k) a[k] = cmulc(a[k], w[k]);
                dft<R, true>(a);
            }
#pragma unroll
            for (int q = 0; q < R; ++q) st(base + q * m, a[q]);
        }
    }
}

template <bool INV, typename LD, typename ST>
__device__ __forceinline__ void stage_warp_any(int r, int P, int m, int Lw, const Tw<1> tw, LD& ld, ST& st,
                                               const float2* ds) {
    switch (r) {
        case 4: stage_warp<4, INV>(P, m, Lw, tw, ld, st, ds); break;
        case 2: stage_warp<2, INV>(P, m, Lw, tw, ld, st, ds); break;
        case 3: stage_warp<3, INV>(P, m, Lw, tw, ld, st, ds); break;
        default: stage_warp<5, INV>(P, m, Lw, tw, ld, st, ds); break;
    }
}

template <int R, typename LD, typename ST>
__device__ __forceinline__ void middle_warp(int P, int Lw, const float* __restrict__ lam, LD& ld, ST& st) {
    const int per = Lw / R, ntop = P / Lw;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    for (int B = warp; B < ntop; B += FT / 32) {
        for (int t = lane; t < per; t += 32) {
            const int base = B * Lw + t * R;
            float2 a[R];
#pragma unroll
            for (int q = 0; q < R; ++q) a[q] = ld(base + q);
            dft<R, false>(a);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const float l = __ldg(&lam[base + q]);
                a[q] = make_float2(a[q].x * l, a[q].y * l);
            }
            dft<R, true>(a);
#pragma unroll
            for (int q = 0; q < R; ++q) st(base + q, a[q]);
        }
    }
}

template <typename LD, typename ST>
__device__ __forceinline__ void middle_warp_any(int r, int P, int Lw, const float* lam, LD& ld, ST& st) {
    switch (r) {
        case 4: middle_warp<4>(P, Lw, lam, ld, st); break;
        case 2: middle_warp<2>(P, Lw, lam, ld, st); break;
        case 3: middle_warp<3>(P, Lw, lam, ld, st); break;
        default: middle_warp<5>(P, Lw, lam, ld, st); break;
    }
}

// barrier after a stage: the warp's when it and the next stage are both warp-local
__device__ __forceinline__ void warp_or_block_sync(bool warp_only) {
    if (warp_only) __syncwarp();
    else __syncthreads();
}

// Position p of the transform: this CTA's shared memory (offset p / C; the
// caller guarantees p = rank mod C) ...
template <int C>
struct SmemLd {
    const float2* buf;
    __device__ __forceinline__ float2 operator()(int p) const { return buf[p >> log2c<C>()]; }
};
template <int C>
struct SmemSt {
    float2* buf;
    __device__ __forceinline__ void operator()(int p, float2 v) const { buf[p >> log2c<C>()] = v; }
};
// ... or the shared memory of CTA p mod C of the cluster
template <int C>
struct ClLd {
    uint32_t base;   // shared-window address of the transform in this CTA
    __device__ __forceinline__ float2 operator()(int p) const {
        return cl_ld(cl_map(base + 8u * (uint32_t)(p >> log2c<C>()), (uint32_t)(p & (C - 1))));
    }
};
template <int C>
struct ClSt {
    uint32_t base;
    __device__ __forceinline__ void operator()(int p, float2 v) const {
        cl_st(cl_map(base + 8u * (uint32_t)(p >> log2c<C>()), (uint32_t)(p & (C - 1))), v);
    }
};

// shared memory of one FFT CTA: its share of the transform and the two twiddle tables
__host__ __device__ inline int64_t tw_hi_entries(int64_t P, int C) {
    const int lo = C == 1 ? TwCfg<1>::LO : TwCfg<2>::LO;
    return (P + lo - 1) / lo;
}
__host__ __device__ inline int64_t tw_lo_entries(int C) { return C == 1 ? TwCfg<1>::PADDED : TwCfg<2>::PADDED; }

// Twiddle tables into shared memory right after this CTA's P / C values of buf.
template <int C>
__device__ Tw<C> load_twiddles(float2* buf, const FftArgs& a) {
    float2* thi = buf + a.P / C;
    float2* tlo = thi + tw_hi_entries(a.P, C);
    constexpr int LO = TwCfg<C>::LO;
    for (int64_t k = threadIdx.x; k * LO < a.P; k += FT) thi[k] = a.tw[k * LO];
    for (int j = threadIdx.x; j < LO; j += FT) tlo[lo_slot(j)] = (j < a.P) ? a.tw[j] : make_float2(1.f, 0.f);
    if constexpr (C == 1) {   // the stages' direct tables, after the two-level ones
        float2* td = tlo + tw_lo_entries(C);
        for (int j = threadIdx.x; j < a.dtw_total; j += FT) td[j] = a.dtw[j];
    }
    return Tw<C>{thi, tlo};
}

// this CTA's shared-memory copy of stage s's direct twiddle table, or NULL
__device__ __forceinline__ const float2* stage_table(const float2* buf, const FftArgs& a, int s) {
    return a.dtw_off[s] < 0 ? nullptr : buf + a.P + tw_hi_entries(a.P, 1) + tw_lo_entries(1) + a.dtw_off[s];
}

// Sum of v over the block (all threads receive it). `scratch` holds 32 floats.
__device__ float block_sum(float v, float* scratch) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    float t = (l < FT / 32) ? scratch[l] : 0.f;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// Sums of v[k] over the trajectory's CTAs (all threads of all of them receive
// them): block sums, then the C partial sums added in rank order, so every CTA
// holds the same bits. xch: K floats of shared memory.
template <int C, int K>
__device__ void traj_sums(float (&v)[K], float* scratch, float* xch) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = block_sum(v[k], scratch);
    if constexpr (C > 1) {
        if (threadIdx.x == 0)
            for (int k = 0; k < K; ++k) xch[k] = v[k];
        cl_sync();
        const uint32_t xa = smem_addr(xch);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float t = 0.f;
            for (int r = 0; r < C; ++r) t += cl_ldf(cl_map(xa + 4u * (uint32_t)k, (uint32_t)r));
            v[k] = t;
        }
        cl_sync();   // every CTA has read the partial sums before any of them moves on
    }
}

__device__ __forceinline__ bool stage_local(const FftArgs& a, int s) { return (a.local_mask >> s) & 1u; }

// P * (C v) for the circulant C with spectrum lam (digit-reversed order), v read
// by `in(position)` (zero beyond the vector) and the result handed to
// `out(position, value)`; `after_first` runs after the first stage (all threads,
// may synchronise), `before_last` before the last one. buf holds this CTA's share
// of the transform and, after it, the twiddle tables.
template <int C, typename IN, typename OUT, typename F1, typename F2>
__device__ __forceinline__ void circulant_io(float2* buf, const FftArgs& a, int rank, IN& in, OUT& out,
                                             F1 after_first, F2 before_last) {
    const Tw<C> tw = load_twiddles<C>(buf, a);
    SmemLd<C> sld{buf};
    SmemSt<C> sst{buf};
    ClLd<C> cld{smem_addr(buf)};
    ClSt<C> cst{smem_addr(buf)};
    const int P = (int)a.P, nst = a.nst;
    __syncthreads();
    if (nst == 1) {   // P <= 5: one CTA
        after_first();
        before_last();
        middle_any<C>(a.radix[0], P, a.lam, in, out, rank);
        return;
    }
    int m = P;
    if constexpr (C == 1) {
        // one CTA: stages from wl on (the middle pass included) run warp by warp
        const int wl = a.wl, Lw = a.Lw;
        for (int s = 0; s + 1 < nst; ++s) {
            m /= a.radix[s];
            const float2* ds = stage_table(buf, a, s);
            if (s == 0) stage_any<false, C>(a.radix[s], P, m, tw, in, sst, rank, ds);
            else if (s >= wl) stage_warp_any<false>(a.radix[s], P, m, Lw, tw, sld, sst, ds);
            else stage_any<false, C>(a.radix[s], P, m, tw, sld, sst, rank, ds);
            warp_or_block_sync(s >= wl);
            if (s == 0) after_first();
        }
        if (nst - 1 >= wl) middle_warp_any(a.radix[nst - 1], P, Lw, a.lam, sld, sst);
        else middle_any<C>(a.radix[nst - 1], P, a.lam, sld, sst, rank);
        warp_or_block_sync(nst - 2 >= wl);
        m = a.radix[nst - 1];
        for (int s = nst - 2; s >= 0; --s) {
            const float2* ds = stage_table(buf, a, s);
            if (s == 0) {
                before_last();
                stage_any<true, C>(a.radix[s], P, m, tw, sld, out, rank, ds);
            } else if (s >= wl) {
                stage_warp_any<true>(a.radix[s], P, m, Lw, tw, sld, sst, ds);
            } else {
                stage_any<true, C>(a.radix[s], P, m, tw, sld, sst, rank, ds);
            }
            m *= a.radix[s];
            warp_or_block_sync(s - 1 >= wl);
        }
        return;
    }
    for (int s = 0; s + 1 < nst; ++s) {
        m /= a.radix[s];
        const bool loc = stage_local(a, s);
        if (s == 0) {
            if (loc) stage_any<false, C>(a.radix[s], P, m, tw, in, sst, rank);
            else stage_any<false, C>(a.radix[s], P, m, tw, in, cst, rank);
        } else {
            if (loc) stage_any<false, C>(a.radix[s], P, m, tw, sld, sst, rank);
            else stage_any<false, C>(a.radix[s], P, m, tw, cld, cst, rank);
        }
        stage_sync<C>(!(loc && stage_local(a, s + 1)));
        if (s == 0) after_first();
    }
    // the middle pass (stride 1): local only for one CTA
    middle_any<C>(a.radix[nst - 1], P, a.lam, cld, cst, rank);
    stage_sync<C>(true);
    m = a.radix[nst - 1];
    for (int s = nst - 2; s >= 0; --s) {
        const bool loc = stage_local(a, s);
        if (s == 0) {
            before_last();
            if (loc) stage_any<true, C>(a.radix[s], P, m, tw, sld, out, rank);
            else stage_any<true, C>(a.radix[s], P, m, tw, cld, out, rank);
        } else {
            if (loc) stage_any<true, C>(a.radix[s], P, m, tw, sld, sst, rank);
            else stage_any<true, C>(a.radix[s], P, m, tw, cld, cst, rank);
        }
        m *= a.radix[s];
        stage_sync<C>(!(loc && (s == 0 || stage_local(a, s - 1))));
    }
}

// First-stage input: s^x + i s^y of one trajectory (zero beyond N), summing
// S^x, S^y on the way.
struct StateIn {
    const float *X, *Y;
    int N;
    float sx = 0.f, sy = 0.f;
    __device__ __forceinline__ float2 operator()(int p) {
        if (p >= N) return make_float2(0.f, 0.f);
        const float2 v = make_float2(__ldg(&X[p]), __ldg(&Y[p]));
        sx += v.x;
        sy += v.y;
        return v;
    }
};

// Predictor at site i from P (W s)_i (Eq. S1; every rounding spelled out): Heun's
// s~, or the midpoint state of the semi-implicit scheme's predictor rotation.
struct PredOut {
    const FftArgs* a;
    int64_t off;
    float Sx = 0.f, Sy = 0.f, inv = 0.f, hdt = 0.f;
    __device__ __forceinline__ void operator()(int i, float2 pf) const {
        if (i >= a->N) return;
        const int64_t e = off + i;
        const float x = a->X[e], y = a->Y[e], z = a->Z[e];
        // B^a = 1/2 (G S^a - (W s^a)_i) dt + noise part; f = s x (B^y, -B^x, 0)
        const float Bx = fmaf(fmaf(a->G, Sx, -__fmul_rn(pf.x, inv)), hdt, a->Bnx[e]);
        const float By = fmaf(fmaf(a->G, Sy, -__fmul_rn(pf.y, inv)), hdt, a->Bny[e]);
        if (a->integ == TWA_INT_MIDPOINT) {
            float mx, my, mz;
            mid_rotation_f32(x, y, z, Bx, By, mx, my, mz);
            a->oX[e] = mx;
            a->oY[e] = my;
            a->oZ[e] = mz;
            return;
        }
        const float fx = __fmul_rn(z, Bx), fy = __fmul_rn(z, By);
        const float fz = -fmaf(x, Bx, __fmul_rn(y, By));
        a->oX[e] = __fadd_rn(x, fx);
        a->oY[e] = __fadd_rn(y, fy);
        a->oZ[e] = __fadd_rn(z, fz);
    }
};

// Corrector and renormalisation at site i; sums of the new state. Heun: from s~
// (X) and s (X0); midpoint scheme: the field of the midpoint state (X) rotates s.
struct CorrOut {
    const FftArgs* a;
    int64_t off;
    float Sx = 0.f, Sy = 0.f, inv = 0.f, hdt = 0.f;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    unsigned bad = 0;
    __device__ __forceinline__ void operator()(int i, float2 pf) {
        if (i >= a->N) return;
        const int64_t e = off + i;
        const float x = a->X[e], y = a->Y[e], z = a->Z[e];
        const float Bx = fmaf(fmaf(a->G, Sx, -__fmul_rn(pf.x, inv)), hdt, a->Bnx[e]);
        const float By = fmaf(fmaf(a->G, Sy, -__fmul_rn(pf.y, inv)), hdt, a->Bny[e]);
        float nx, ny, nz;
        if (a->integ == TWA_INT_MIDPOINT) {
            // s' = 2 m - s of the rotation of s by the midpoint field
            const float s0x = a->X0[e], s0y = a->Y0[e], s0z = a->Z0[e];
            float mx, my, mz;
            mid_rotation_f32(s0x, s0y, s0z, Bx, By, mx, my, mz);
            nx = fmaf(2.0f, mx, -s0x);
            ny = fmaf(2.0f, my, -s0y);
            nz = fmaf(2.0f, mz, -s0z);
        } else {
            // s' = (s + s~)/2 + f(s~)/2, then |s'| = sqrt(3)
            const float hx = __fmul_rn(0.5f, __fadd_rn(a->X0[e], x));
            const float hy = __fmul_rn(0.5f, __fadd_rn(a->Y0[e], y));
            const float hz = __fmul_rn(0.5f, __fadd_rn(a->Z0[e], z));
            nx = fmaf(0.5f, __fmul_rn(z, Bx), hx);
            ny = fmaf(0.5f, __fmul_rn(z, By), hy);
            nz = fmaf(-0.5f, fmaf(x, Bx, __fmul_rn(y, By)), hz);
        }
        if (a->renorm) {
            const float s = sqrtf(3.0f / fmaf(nx, nx, fmaf(ny, ny, __fmul_rn(nz, nz))));
            nx = __fmul_rn(nx, s);
            ny = __fmul_rn(ny, s);
            nz = __fmul_rn(nz, s);
        }
        if (!(isfinite(nx) && isfinite(ny) && isfinite(nz))) ++bad;
        a->oX[e] = nx;
        a->oY[e] = ny;
        a->oZ[e] = nz;
        sx += nx;
        sy += ny;
        sz += nz;
    }
};

template <int C>
__global__ void __launch_bounds__(FT, 1) k_fft_pred(const __grid_constant__ FftArgs a) {
    extern __shared__ float2 buf[];
    __shared__ float scratch[32];
    __shared__ float xch[4];
    const int rank = cl_rank<C>();
    const int64_t off = (int64_t)(blockIdx.x / C) * a.N;
    StateIn in{a.X + off, a.Y + off, (int)a.N};
    PredOut out{&a, off};
    out.inv = 1.0f / (float)a.P;
    out.hdt = 0.5f * a.dt;
    auto first = [&]() {
        if (a.nst == 1)
            for (int p = threadIdx.x; p < a.N; p += FT) in(p);   // sums only (tiny P)
        float v[2] = {in.sx, in.sy};
        traj_sums<C>(v, scratch, xch);
        out.Sx = v[0];
        out.Sy = v[1];
        in.sx = in.sy = 0.f;
    };
    circulant_io<C>(buf, a, rank, in, out, first, [] {});
}

template <int C>
__global__ void __launch_bounds__(FT, 1) k_fft_corr(const __grid_constant__ FftArgs a) {
    extern __shared__ float2 buf[];
    __shared__ float scratch[32];
    __shared__ float xch[4];
    const int rank = cl_rank<C>();
    const int64_t m = blockIdx.x / C, off = m * a.N;
    const int64_t t1 = *a.d_t + 1;
    StateIn in{a.X + off, a.Y + off, (int)a.N};
    CorrOut out{&a, off};
    out.inv = 1.0f / (float)a.P;
    out.hdt = 0.5f * a.dt;
    auto first = [&]() {
        if (a.nst == 1)
            for (int p = threadIdx.x; p < a.N; p += FT) in(p);
        float v[2] = {in.sx, in.sy};
        traj_sums<C>(v, scratch, xch);
        out.Sx = v[0];
        out.Sy = v[1];
        in.sx = in.sy = 0.f;
    };
    circulant_io<C>(buf, a, rank, in, out, first, [] {});
    float v[3] = {out.sx, out.sy, out.sz};
    traj_sums<C>(v, scratch, xch);
    const float Sx = v[0], Sy = v[1], Sz = v[2];
    const unsigned nb = __reduce_add_sync(0xffffffffu, out.bad);
    if ((threadIdx.x & 31) == 0 && nb) atomicAdd(&a.flags[FLAG_NONFINITE], (unsigned long long)nb);
    if (threadIdx.x == 0 && rank == 0) {
        if (window_sample(t1, a.n_window, a.n_stride)) {
            // window moments S^z, A, A^2, A S^z, (S^z)^2 with A = ((S^x)^2 + (S^y)^2) / 4
            const double dx = Sx, dy = Sy, dz = Sz;
            const double A = 0.25 * (dx * dx + dy * dy);
            double* mm = a.mom + 5 * m;
            mm[0] += dz;
            mm[1] += A;
            mm[2] += A * A;
            mm[3] += A * dz;
            mm[4] += dz * dz;
        }
        __threadfence();
        const unsigned long long done = atomicAdd(&a.flags[FLAG_DONE], 1ull);
        if (done == gridDim.x / C - 1) {   // last trajectory of the step: advance the counter
            a.flags[FLAG_DONE] = 0ull;
            if (window_sample(t1, a.n_window, a.n_stride)) *a.d_count += 1;
            __threadfence();
            *a.d_t = t1;
        }
    }
}

// Circulant draw of the pump noise of step t = *d_t for trajectory m: position p
// of the inverse transform's input holds sqrt(lam_k / P) (a_k + i b_k), k its
// frequency, (a_k, b_k) the FP32 Box-Muller pair of Philox counter (m, t, k, 2);
// the transform returns Y_j in natural order, chi^x_j = Re Y_j, chi^y_j = Im Y_j.
// Writes the noise part of the field increment, sqrt(G dt) xi^a - sqrt(dt) chi^a_j,
// xi^a the collective normals of counter (m, t, N, 0). The draws are made in the
// first inverse stage and the noise part written by the last one.
struct NoiseIn {
    const float* nscale;
    const int32_t* nfreq;
    uint64_t seed;
    uint32_t m, t;
    __device__ __forceinline__ float2 operator()(int p) const {
        float ga, gb;
        normal2_f32(seed, m, t, (uint32_t)__ldg(&nfreq[p]), ga, gb, STREAM_CIRCULANT);
        const float sc = __ldg(&nscale[p]);
        return make_float2(__fmul_rn(sc, ga), __fmul_rn(sc, gb));
    }
};
struct NoiseOut {
    float *Bnx, *Bny;
    int N;
    float nx0, ny0, sdt;
    __device__ __forceinline__ void operator()(int j, float2 y) const {
        if (j >= N) return;
        Bnx[j] = fmaf(-sdt, y.x, nx0);
        Bny[j] = fmaf(-sdt, y.y, ny0);
    }
};

template <int C>
__global__ void __launch_bounds__(FT, 1) k_fft_noise(const __grid_constant__ FftArgs a, const float* nscale,
                                                     const int32_t* nfreq, uint64_t seed, int64_t m0, float sgdt,
                                                     float sdt, float* Bnx, float* Bny) {
    extern __shared__ float2 buf[];
    const int rank = cl_rank<C>();
    const int64_t m = blockIdx.x / C, off = m * a.N;
    const uint32_t t = (uint32_t)(*a.d_t), mg = (uint32_t)(m0 + m);
    const Tw<C> tw = load_twiddles<C>(buf, a);
    float xi_x, xi_y;
    normal2_f32(seed, mg, t, (uint32_t)a.N, xi_x, xi_y);
    NoiseIn in{nscale, nfreq, seed, mg, t};
    NoiseOut out{Bnx + off, Bny + off, (int)a.N, __fmul_rn(sgdt, xi_x), __fmul_rn(sgdt, xi_y), sdt};
    SmemLd<C> sld{buf};
    SmemSt<C> sst{buf};
    ClLd<C> cld{smem_addr(buf)};
    ClSt<C> cst{smem_addr(buf)};
    const int P = (int)a.P, nst = a.nst;
    // every CTA of the cluster is running before the first stage writes into them
    stage_sync<C>(true);
    // unnormalised inverse transform, digit-reversed input -> natural order
    int mm = 1;
    if constexpr (C == 1) {
        // stages from wl on run warp by warp (the first stage reads global memory)
        const int wl = a.wl, Lw = a.Lw;
        for (int s = nst - 1; s >= 0; --s) {
            const float2* ds = stage_table(buf, a, s);
            if (s == nst - 1 && s == 0) stage_any<true, C>(a.radix[s], P, mm, tw, in, out, rank, ds);
            else if (s == 0) stage_any<true, C>(a.radix[s], P, mm, tw, sld, out, rank, ds);
            else if (s >= wl && s == nst - 1) stage_warp_any<true>(a.radix[s], P, mm, Lw, tw, in, sst, ds);
            else if (s >= wl) stage_warp_any<true>(a.radix[s], P, mm, Lw, tw, sld, sst, ds);
            else if (s == nst - 1) stage_any<true, C>(a.radix[s], P, mm, tw, in, sst, rank, ds);
            else stage_any<true, C>(a.radix[s], P, mm, tw, sld, sst, rank, ds);
            mm *= a.radix[s];
            warp_or_block_sync(s - 1 >= wl);
        }
        return;
    }
    for (int s = nst - 1; s >= 0; --s) {
        const bool loc = stage_local(a, s);
        if (s == nst - 1 && s == 0) stage_any<true, C>(a.radix[s], P, mm, tw, in, out, rank);
        else if (s == nst - 1) {
            if (loc) stage_any<true, C>(a.radix[s], P, mm, tw, in, sst, rank);
            else stage_any<true, C>(a.radix[s], P, mm, tw, in, cst, rank);
        } else if (s == 0) {
            if (loc) stage_any<true, C>(a.radix[s], P, mm, tw, sld, out, rank);
            else stage_any<true, C>(a.radix[s], P, mm, tw, cld, out, rank);
        } else {
            if (loc) stage_any<true, C>(a.radix[s], P, mm, tw, sld, sst, rank);
            else stage_any<true, C>(a.radix[s], P, mm, tw, cld, cst, rank);
        }
        mm *= a.radix[s];
        stage_sync<C>(!(loc && (s == 0 || stage_local(a, s - 1))));
    }
}

// W s for caller vectors: vectors 2b and 2b+1 share one complex transform.
struct FieldIn {
    const double *v0, *v1;   // v1 NULL for an odd last vector
    int N;
    __device__ __forceinline__ float2 operator()(int p) const {
        if (p >= N) return make_float2(0.f, 0.f);
        return make_float2((float)v0[p], v1 ? (float)v1[p] : 0.f);
    }
};
struct FieldOut {
    double *o0, *o1;
    int N;
    double inv;
    __device__ __forceinline__ void operator()(int p, float2 v) const {
        if (p >= N) return;
        o0[p] = (double)v.x * inv;
        if (o1) o1[p] = (double)v.y * inv;
    }
};

template <int C>
__global__ void __launch_bounds__(FT, 1) k_fft_field(const __grid_constant__ FftArgs a) {
    extern __shared__ float2 buf[];
    const int rank = cl_rank<C>();
    const int64_t k0 = 2 * (int64_t)(blockIdx.x / C), k1 = k0 + 1;
    const bool two = k1 < a.K;
    FieldIn in{a.field_in + k0 * a.N, two ? a.field_in + k1 * a.N : nullptr, (int)a.N};
    FieldOut out{a.field_out + k0 * a.N, two ? a.field_out + k1 * a.N : nullptr, (int)a.N, 1.0 / (double)a.P};
    circulant_io<C>(buf, a, rank, in, out, [] {}, [] {});
}

// exp(-2 pi i n / P), accurate to FP32 rounding (FP64 sincospi).
__global__ void k_fft_twiddles(float2* tw, int64_t P) {
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= P) return;
    double s, c;
    sincospi(2.0 * (double)n / (double)P, &s, &c);
    tw[n] = make_float2((float)c, (float)-s);
}

struct RadixPlan {
    int nst;
    int radix[40];
};

// First column of the embedding on the circle of length P, for d <= P / 2:
// c_d = w / (1 + d)^alpha (the expression of the pump-matrix kernel).
__global__ void k_fft_sequence(double* cseq, int64_t P, double alpha, double w) {
    const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (d > P / 2) return;
    double v;
    if (isinf(alpha)) v = (d == 0) ? w : 0.0;
    else if (alpha == 0.0) v = w;
    else v = w / pow((double)(d + 1), alpha);
    cseq[d] = v;
}

// Spectrum lam_k = c_0 + 2 sum_{0<d<P/2} c_d cos(2 pi k d / P) + c_{P/2} (-1)^k
// in FP64, written at the DIF output position p of frequency k (mixed-radix
// digit reversal), with the noise-draw scale sqrt(max(lam_k, 0) / P) and k.
__global__ void k_fft_lambda(float* lam, float* nscale, int32_t* nfreq, const double* cseq, int64_t P,
                             const RadixPlan plan) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    int64_t rem = p, span = P, k = 0, weight = 1;
    for (int s = 0; s < plan.nst; ++s) {
        span /= plan.radix[s];
        const int64_t ks = rem / span;
        rem -= ks * span;
        k += ks * weight;
        weight *= plan.radix[s];
    }
    const int64_t h = P / 2;
    double acc = cseq[0] + ((k & 1) ? -cseq[h] : cseq[h]);
    int64_t r = 0;   // k d mod P, advanced by k each term (k < P)
    for (int64_t d = 1; d < h; ++d) {
        r += k;
        if (r >= P) r -= P;
        acc += 2.0 * cseq[d] * cospi(2.0 * (double)r / (double)P);
    }
    lam[p] = (float)acc;
    nscale[p] = (float)sqrt(fmax(acc, 0.0) / (double)P);
    nfreq[p] = (int32_t)k;
}

bool smooth(int64_t v) {
    for (int f : {2, 3, 5})
        while (v % f == 0) v /= f;
    return v == 1;
}

FftArgs base_args(twa_ctx* c) {
    FftArgs a{};
    const FftPlan* f = c->fft;
    a.N = c->N;
    a.M = c->M;
    a.P = f->P;
    a.nst = f->nst;
    for (int s = 0; s < f->nst; ++s) a.radix[s] = f->radix[s];
    a.local_mask = f->local_mask;
    a.wl = f->wl;
    a.Lw = (int)f->Lw;
    a.dtw = f->dtw;
    a.dtw_total = (int)f->dtw_total;
    for (int k = 0; k < 40; ++k) a.dtw_off[k] = f->dtw_off[k];
    a.lam = f->lam;
    a.tw = f->tw;
    a.G = (float)c->Gamma;
    a.dt = (float)c->dt;
    a.renorm = c->opts.renormalize;
    a.integ = c->opts.integrator;
    a.flags = c->d_flags;
    return a;
}

// shared memory of one FFT CTA: its share of the transform and the two twiddle tables
size_t smem_bytes(int64_t P, int C) {
    return sizeof(float2) * (size_t)(P / C + tw_hi_entries(P, C) + tw_lo_entries(C));
}
// ... and the direct tables of the plan's stages
size_t plan_smem(const FftPlan* f) { return smem_bytes(f->P, f->C) + sizeof(float2) * (size_t)f->dtw_total; }

// dtw[off_s + j] = w^(j P / L_s) = exp(-2 pi i j / L_s), from the full table tw
__global__ void k_fft_stage_tables(float2* dtw, const float2* tw, const int64_t* off, const int64_t* step,
                                   const int64_t* len, int nst) {
    for (int s = 0; s < nst; ++s) {
        if (off[s] < 0) continue;
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len[s]; j += (int64_t)gridDim.x * blockDim.x)
            dtw[off[s] + j] = tw[j * step[s]];
    }
}

// Call f with the cluster size as a compile-time constant.
template <typename F>
int with_c(int C, F f) {
    switch (C) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        default: return f(std::integral_constant<int, 8>{});
    }
}

// One CTA per unit (trajectory, vector pair), or one cluster of C CTAs per unit.
template <typename... KArgs, typename... Args>
int fft_launch(twa_ctx* c, void (*kern)(KArgs...), int64_t units, Args... args) {
    const int C = c->fft->C;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(units * C));
    cfg.blockDim = dim3(FT);
    cfg.dynamicSmemBytes = plan_smem(c->fft);
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = C > 1 ? 1 : 0;
    TWA_CUDA(c, cudaLaunchKernelEx(&cfg, kern, args...));
    return TWA_OK;
}

template <int C>
int set_smem(twa_ctx* c) {
    const void* ks[] = {(const void*)k_fft_pred<C>, (const void*)k_fft_corr<C>, (const void*)k_fft_field<C>,
                        (const void*)k_fft_noise<C>};
    const int bytes = (int)plan_smem(c->fft);
    for (const void* k : ks) TWA_CUDA(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    if (C > 1) {   // the cluster must fit: C SMs of one GPC, each holding one such CTA
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(FT);
        cfg.dynamicSmemBytes = (size_t)bytes;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        TWA_CUDA(c, cudaOccupancyMaxActiveClusters(&n, (const void*)k_fft_corr<C>, &cfg));
        if (n < 1) return set_error(c, TWA_EUNSUPPORTED, "FFT route: no cluster of " + std::to_string(C) + " CTAs fits");
    }
    return TWA_OK;
}

int env_int(const char* name, int dflt) {
    const char* v = getenv(name);
    return v ? atoi(v) : dflt;
}

}  // namespace

int fft_prepare(twa_ctx* c) {
    const int64_t need = 2 * c->N - 2 > 2 ? 2 * c->N - 2 : 2;
    int max_smem = 0;
    TWA_CUDA(c, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    // the transform in one CTA while it fits its shared memory, else in the
    // smallest cluster that holds it; TWA_FFT_CLUSTER = 1, 2, 4 or 8 forces the size
    const int forced = env_int("TWA_FFT_CLUSTER", 0);
    if (forced && forced != 1 && forced != 2 && forced != 4 && forced != 8)
        return set_error(c, TWA_EINVAL, "TWA_FFT_CLUSTER must be 1, 2, 4 or 8");
    int C = 0;
    int64_t P = 0;
    for (int cc = 1; cc <= FFT_MAX_C; cc *= 2) {
        if (forced && cc != forced) continue;
        // smallest 2^a 3^b 5^c >= need that is even (one CTA) or a multiple of 4 C
        // (a cluster: every stage's butterfly count then divides among its CTAs)
        const int64_t q = cc == 1 ? 2 : 4 * cc;
        int64_t p = need;
        while (p % q || !smooth(p)) ++p;
        if (p / cc <= FFT_MAX_PLOC && smem_bytes(p, cc) <= (size_t)max_smem) {
            C = cc;
            P = p;
            break;
        }
    }
    if (!C)
        return set_error(c, TWA_EUNSUPPORTED, "FFT route: the transform for N = " + std::to_string((long long)c->N) +
                                                  " does not fit the shared memory of a cluster of " +
                                                  std::to_string(forced ? forced : FFT_MAX_C) + " CTAs");
    FftPlan* f = new FftPlan();
    c->fft = f;
    f->P = P;
    f->C = C;
    int64_t v = P;
    f->nst = 0;
    if (C == 1) {   // radices 4, (2), 3, 5
        while (v % 4 == 0) { f->radix[f->nst++] = 4; v /= 4; }
        while (v % 2 == 0) { f->radix[f->nst++] = 2; v /= 2; }
        while (v % 3 == 0) { f->radix[f->nst++] = 3; v /= 3; }
        while (v % 5 == 0) { f->radix[f->nst++] = 5; v /= 5; }
    } else {        // radices 5, 3, (2), 4: the powers of two last, so the strides stay multiples of C
        while (v % 5 == 0) { f->radix[f->nst++] = 5; v /= 5; }
        while (v % 3 == 0) { f->radix[f->nst++] = 3; v /= 3; }
        int two = 0;   // v = 2^two now
        for (int64_t t = v; t > 1; t /= 2) ++two;
        if (two % 2) { f->radix[f->nst++] = 2; v /= 2; }
        while (v % 4 == 0) { f->radix[f->nst++] = 4; v /= 4; }
    }
    // one CTA: the first stage s >= 1 with at least 32 blocks (span P / (r_0 ... r_{s-1}))
    // that 32 warps share evenly enough (the busiest warp at most 1.25x the mean)
    // runs, with every later stage, warp by warp (TWA_FFT_WARP = 0: no such stage)
    f->wl = f->nst;
    f->Lw = 0;
    if (C == 1 && env_int("TWA_FFT_WARP", 1) != 0) {
        int64_t L = P;
        for (int s = 0; s < f->nst; ++s) {
            const int64_t ntop = P / L;
            if (s >= 1 && ntop >= 32 && (ntop + 31) / 32 * 32 * 4 <= ntop * 5) {
                f->wl = s;
                f->Lw = L;
                break;
            }
            L /= f->radix[s];
        }
    }
    // stage s has stride m_s = P / (r_0 ... r_s); it stays inside one CTA when C divides m_s
    f->local_mask = 0;
    for (int64_t s = 0, m = P; s < f->nst; ++s) {
        m /= f->radix[s];
        if (m % C == 0) f->local_mask |= 1u << s;
    }
    Scratch<double> cseq_buf(c, c->stream);
    if (dev_malloc(c, &f->lam, sizeof(float) * P) != cudaSuccess ||
        dev_malloc(c, &f->tw, sizeof(float2) * P) != cudaSuccess ||
        dev_malloc(c, &f->nscale, sizeof(float) * P) != cudaSuccess ||
        dev_malloc(c, &f->nfreq, sizeof(int32_t) * P) != cudaSuccess ||
        cseq_buf.alloc(sizeof(double) * (P / 2 + 1)) != cudaSuccess)
        return set_error(c, TWA_ENOMEM, "device allocation of the FFT plan");
    double* cseq = cseq_buf.p;
    RadixPlan rp{};
    rp.nst = f->nst;
    for (int s = 0; s < f->nst; ++s) rp.radix[s] = f->radix[s];
    const unsigned g = (unsigned)((P + 255) / 256);
    k_fft_twiddles<<<g, 256, 0, c->stream>>>(f->tw, P);
    k_fft_sequence<<<(unsigned)((P / 2 + 256) / 256), 256, 0, c->stream>>>(cseq, P, c->alpha, c->w);
    k_fft_lambda<<<g, 256, 0, c->stream>>>(f->lam, f->nscale, f->nfreq, cseq, P, rp);
    TWA_CUDA(c, cudaGetLastError());
    // one CTA: direct twiddle tables for the stages, smallest first, while they fit
    // the shared memory beside the transform (TWA_FFT_DIRECT_TW = 0: none)
    for (int s = 0; s < 40; ++s) f->dtw_off[s] = -1;
    f->dtw_total = 0;
    if (C == 1 && f->nst > 1 && env_int("TWA_FFT_DIRECT_TW", 1) != 0) {
        std::vector<int64_t> off(f->nst, -1), step(f->nst, 0), len(f->nst, 0);
        std::vector<int64_t> ms(f->nst);
        for (int64_t s = 0, m = P; s < f->nst; ++s) ms[s] = (m /= f->radix[s]);
        // (1 KB kept back for the kernels' static shared memory)
        const int64_t room = ((int64_t)max_smem - 1024 - (int64_t)smem_bytes(P, 1)) / (int64_t)sizeof(float2);
        for (int s = f->nst - 2; s >= 0; --s) {   // the middle stage (stride 1) has no twiddles
            if (f->dtw_total + ms[s] > room) break;
            off[s] = f->dtw_total;
            len[s] = ms[s];
            step[s] = P / (ms[s] * f->radix[s]);
            f->dtw_off[s] = (int)f->dtw_total;
            f->dtw_total += ms[s];
        }
        if (f->dtw_total > 0) {
            Scratch<int64_t> meta(c, c->stream);
            if (dev_malloc(c, &f->dtw, sizeof(float2) * f->dtw_total) != cudaSuccess ||
                meta.alloc(sizeof(int64_t) * 3 * f->nst) != cudaSuccess)
                return set_error(c, TWA_ENOMEM, "device allocation of the FFT plan");
            std::vector<int64_t> h(3 * f->nst);
            for (int s = 0; s < f->nst; ++s) {
                h[s] = off[s];
                h[f->nst + s] = step[s];
                h[2 * f->nst + s] = len[s];
            }
            TWA_CUDA(c, cudaMemcpyAsync(meta.p, h.data(), sizeof(int64_t) * h.size(), cudaMemcpyHostToDevice,
                                        c->stream));
            k_fft_stage_tables<<<64, 256, 0, c->stream>>>(f->dtw, f->tw, meta.p, meta.p + f->nst,
                                                          meta.p + 2 * f->nst, f->nst);
            TWA_CUDA(c, cudaGetLastError());
            TWA_CUDA(c, cudaStreamSynchronize(c->stream));   // h and meta live until here
        }
    }
    return with_c(C, [&](auto cc) { return set_smem<decltype(cc)::value>(c); });
}

void fft_free(twa_ctx* c) {
    if (!c->fft) return;
    void* p[] = {c->fft->lam, c->fft->tw, c->fft->nscale, c->fft->nfreq, c->fft->dtw};
    for (void* q : p) dev_free(c, q);
    delete c->fft;
    c->fft = nullptr;
}

int fft_predict(twa_ctx* c) {
    TcState* t = c->tc;
    FftArgs a = base_args(c);
    a.X = t->X; a.Y = t->Y; a.Z = t->Z;
    a.Bnx = t->Bx; a.Bny = t->By;
    a.oX = t->Xp; a.oY = t->Yp; a.oZ = t->Zp;
    return with_c(c->fft->C, [&](auto cc) { return fft_launch(c, k_fft_pred<decltype(cc)::value>, c->M, a); });
}

int fft_correct(twa_ctx* c) {
    TcState* t = c->tc;
    FftArgs a = base_args(c);
    a.X = t->Xp; a.Y = t->Yp; a.Z = t->Zp;
    a.X0 = t->X; a.Y0 = t->Y; a.Z0 = t->Z;
    a.Bnx = t->Bx; a.Bny = t->By;
    a.oX = t->X; a.oY = t->Y; a.oZ = t->Z;
    a.mom = c->mom;
    a.d_t = c->d_t;
    a.d_count = c->d_count;
    a.n_window = c->n_window;
    a.n_stride = c->n_stride;
    return with_c(c->fft->C, [&](auto cc) { return fft_launch(c, k_fft_corr<decltype(cc)::value>, c->M, a); });
}

int fft_noise(twa_ctx* c) {
    TcState* t = c->tc;
    FftArgs a = base_args(c);
    a.d_t = c->d_t;
    const float* ns = c->fft->nscale;
    const int32_t* nf = c->fft->nfreq;
    const uint64_t seed = c->seed;
    const int64_t m0 = c->opts.traj_offset;
    const float sgdt = (float)sqrt(c->Gamma * c->dt), sdt = (float)sqrt(c->dt);
    float *bx = t->Bx, *by = t->By;
    return with_c(c->fft->C, [&](auto cc) {
        return fft_launch(c, k_fft_noise<decltype(cc)::value>, c->M, a, ns, nf, seed, m0, sgdt, sdt, bx, by);
    });
}

int fft_field(twa_ctx* c, const double* s, double* P, int64_t K) {
    FftArgs a = base_args(c);
    a.field_in = s;
    a.field_out = P;
    a.K = K;
    return with_c(c->fft->C, [&](auto cc) { return fft_launch(c, k_fft_field<decltype(cc)::value>, (K + 1) / 2, a); });
}

}  // namespace twa

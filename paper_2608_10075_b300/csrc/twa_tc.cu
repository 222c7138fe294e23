// Mixed-precision tensor-core path (sm_103a): the per-step contractions of Eq. S1
// -- the pump field sum_j w_ij s^a_j and the correlated noise (L eta)_i -- run as
// tcgen05.mma (kind::f16, BF16 operands, FP32 accumulators in TMEM) on tiles that
// TMA stages into shared memory; the stochastic-Heun update is the epilogue of
// the contraction that needs it.
//
// Operands (K = site index j, contiguous):
//   A = W or L images, [N][ldk] BF16, rows = sites i (MMA M = 128 per tile)
//   B = state / noise images, [2M][ldk] BF16, row 2m = x of trajectory m, row
//       2m+1 = y (MMA N = BN per tile = BN/2 trajectories x (x, y))
// so accumulator column 2j / 2j+1 of a tile holds the x / y contraction of
// trajectory m0 + j at site i0 + lane, and every epilogue thread owns one site.
//
// Precision modes: BF16 (one term, hi*hi) or BF16X3 (hi*hi + hi*lo + lo*hi,
// hi = bf16(v), lo = bf16(v - hi)), FP32 accumulation. The noise eta is drawn
// in FP32 and rounded to BF16 once, so L.eta needs the two terms of L only.
// TF32 (kind::tf32, one term, operands rounded to TF32 in FP32 containers) and
// FP32 (the same split as BF16X3 with hi = tf32(v), lo = tf32(v - hi): about
// 22 significant bits, FP32-accurate contractions; eta split as well, so L.eta
// has three terms) run on a 16-wide FP32 K stage.
//
// Kernel structure: persistent CTAs (at most one per SM) walk a static list of
// (row tile, trajectory tile) pairs, strided or from a host-built schedule.
// Warp 0 streams K tiles through a ring of shared-memory stages with TMA,
// running ahead across tile boundaries; warp 1 issues the MMAs into one of two
// TMEM accumulators; warps 2-17 run the epilogue of the previous tile from the
// other accumulator (four warps per TMEM lane quadrant, each on a quarter of
// the columns), so epilogue and main loop overlap. Every wait on an mbarrier is
// bounded in time and reports a timeout.
//
// A step t is: noise of step t + 1; one launch with the tiles of W.s and the
// Heun predictor plus part of the L.eta tiles of step t + 1 (-> noise part of
// its field increment); one launch with W.s~ and the corrector plus the other
// L.eta tiles; closing kernel (moments). The first step of a run computes its
// own noise part first. Collective sums S^a are passed between kernels as
// per-row-tile partial sums, reduced in a fixed order.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <queue>
#include <type_traits>
#include <vector>

#include <cudaTypedefs.h>

#include "twa_internal.cuh"

namespace twa {

namespace {

constexpr int BM = TC_BM;
// warp 0 TMA, warp 1 MMA, warps 2.. epilogue: EPI_GROUPS per TMEM lane quadrant,
// each draining its share of the accumulator columns, so that more state loads
// are in flight (same-box A/B at N = 1e4: 4 groups 1.6 % faster than 2, which
// were ~6 % faster than 1; batched N = 3000 points gain more)
constexpr int EPI_GROUPS = 4, EPI_WARPS = 4 * EPI_GROUPS, EPI_THREADS = 32 * EPI_WARPS;
constexpr int NTHREADS = 64 + EPI_THREADS;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bounded waits: 2 s

// MODE_MIX: tiles of several modes in one launch, each problem's mode and term
// count read from its group descriptor.
enum Mode { MODE_FIELD = 0, MODE_LETA = 1, MODE_PRED = 2, MODE_CORR = 3, MODE_MIX = 4 };

// K-stage configurations: K tile width (elements), element size, swizzle and ring
// depth. KC = 2 is the TF32 precision mode: FP32 containers holding TF32 values,
// kind::tf32 MMAs (K = 8 per instruction, the same 32 bytes of a row as 16 BF16).
// KC = 3 is KC = 1 for the precisions whose operand has no lo image (at most two
// products per entry): a stage holds A hi, A lo and one B image, 32 KB instead of
// 48 KB, so the ring is six stages deep in the same shared memory.
template <int KC>
struct KCfg;
template <>
struct KCfg<0> {   // 64 BF16 = 128 B rows, SWIZZLE_128B, two stages
    static constexpr int BK = 64, STAGES = 2, ESZ = 2;
    static constexpr bool TF32 = false, ONE_B = false;
    static constexpr uint64_t LAYOUT = 2;   // descriptor layout code of SWIZZLE_128B
    static constexpr uint32_t SBO = 1024;   // 8 rows x 128 B
};
template <>
struct KCfg<1> {   // 32 BF16 = 64 B rows, SWIZZLE_64B, four stages
    static constexpr int BK = 32, STAGES = 4, ESZ = 2;
    static constexpr bool TF32 = false, ONE_B = false;
    static constexpr uint64_t LAYOUT = 4;   // SWIZZLE_64B
    static constexpr uint32_t SBO = 512;    // 8 rows x 64 B
};
template <>
struct KCfg<2> {   // 16 TF32 = 64 B rows, SWIZZLE_64B, four stages
    static constexpr int BK = 16, STAGES = 4, ESZ = 4;
    static constexpr bool TF32 = true, ONE_B = false;
    static constexpr uint64_t LAYOUT = 4;
    static constexpr uint32_t SBO = 512;
};
template <>
struct KCfg<3> {   // 32 BF16 = 64 B rows, SWIZZLE_64B, six stages of A hi, A lo, B
    static constexpr int BK = 32, STAGES = 6, ESZ = 2;
    static constexpr bool TF32 = false, ONE_B = true;
    static constexpr uint64_t LAYOUT = 4;
    static constexpr uint32_t SBO = 512;
};
template <>
struct KCfg<4> {   // 64 BF16 = 128 B rows, SWIZZLE_128B, three stages of A hi, A lo, B
    static constexpr int BK = 64, STAGES = 3, ESZ = 2;
    static constexpr bool TF32 = false, ONE_B = true;
    static constexpr uint64_t LAYOUT = 2;
    static constexpr uint32_t SBO = 1024;
};
// Pair-CTA configurations: the two CTAs of a cluster share one 256-row MMA
// (tcgen05.mma.cta_group::2). Each holds the A rows of its own 128-row tile and
// half of the B rows, so a B image takes half the bytes of a stage and the ring
// is deeper in the same shared memory: A hi, A lo, B hi, B lo halves in six
// stages (KC = 1), A hi, A lo and one B half in eight (KC = 3).
template <int KC, bool PAIR>
struct RingDepth {
    static constexpr int value = KCfg<KC>::STAGES;
};
template <>
struct RingDepth<1, true> {
    static constexpr int value = 6;
};
template <>
struct RingDepth<3, true> {
    static constexpr int value = 8;
};
template <>
struct RingDepth<4, true> {   // 3 x 16 KB
    static constexpr int value = 4;
};
template <>
struct RingDepth<0, true> {   // 4 x 16 KB
    static constexpr int value = 3;
};
inline int kcfg_bk(int kc) { return (kc == 0 || kc == 4) ? 64 : kc == 2 ? KCfg<2>::BK : KCfg<1>::BK; }
// products per L.eta entry: one term, two (L hi + lo against the single BF16 eta
// of BF16X3) or three (FP32 mode: eta split into TF32 hi + lo as well)
inline int leta_terms(const TcState* t) { return t->lterms; }

template <int BN, int KC, bool PAIR = false>
struct Geo {
    static constexpr int BK = KCfg<KC>::BK, STAGES = RingDepth<KC, PAIR>::value;
    static constexpr int BROWS = PAIR ? BN / 2 : BN;   // B rows one CTA holds
    static constexpr int MROWS = PAIR ? 2 * BM : BM;   // M of the MMA
    static constexpr int A_BYTES = BM * BK * KCfg<KC>::ESZ;
    static constexpr int B_BYTES = BROWS * BK * KCfg<KC>::ESZ;
    static constexpr int MMAS = BK * KCfg<KC>::ESZ / 32;   // MMAs per stage: 32 bytes of K each
    static constexpr int STAGE_BYTES = 2 * A_BYTES + (KCfg<KC>::ONE_B ? 1 : 2) * B_BYTES;
    static constexpr int TILES = STAGES * STAGE_BYTES;
    static constexpr int NTRAJ = BN / 2;
    static constexpr int EXTRA = (2 * STAGES + 4) * 8 + 16 + NTRAJ * 2 * 4 * 2 + 4 * NTRAJ * 3 * 4;
    static constexpr int SMEM = TILES + EXTRA + 1024;
    static constexpr uint32_t NCOLS = (2 * BN <= 256) ? 256 : 512;
    // instruction descriptor: D = F32 (bits 4-5 = 1), A and B format at bits 7-9 and
    // 10-12 (kind::f16: BF16 = 1; kind::tf32: TF32 = 2), both K-major, N >> 3 at
    // bits 17-22, M >> 4 at bits 24-28 (M = 256 for a CTA pair).
    static constexpr uint32_t FMT = KCfg<KC>::TF32 ? 2u : 1u;
    static constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(MROWS >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// CL: acquire at cluster scope, for a barrier that threads of the peer CTA
// arrive on remotely
template <bool CL = false>
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    if constexpr (CL) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    }
    return ok != 0;
}

// Wait for the phase with the given parity; gives up after WAIT_NS (or at once
// when another CTA has already given up and `follow_abort` is set), counting the
// timeout in flags[FLAG_TIMEOUT].
template <bool CL = false>
__device__ __noinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long* flags,
                                       bool follow_abort, unsigned long long limit_ns = WAIT_NS) {
    if (mbar_try<CL>(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    volatile unsigned long long* vf = flags;
    while (true) {
        if (mbar_try<CL>(bar, parity)) return true;
        if (follow_abort && vf[FLAG_TIMEOUT] != 0ull) return false;
        if (gtimer() - t0 > limit_ns) {
            atomicAdd(&flags[FLAG_TIMEOUT], 1ull);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// ---- CTA pairs (clusters of two) ----
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the variable at p in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
    return a;
}

// every thread of both CTAs; orders shared-memory accesses across the pair
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}

// TMA load into this CTA's shared memory whose completion is counted on a
// barrier of either CTA of the pair (the leader's: its MMA reads both halves)
__device__ __forceinline__ void tma_load_pair(void* dst, const CUtensorMap* map, uint32_t cluster_bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(cluster_bar), "r"(x), "r"(y)
        : "memory");
}

// 256-row MMA of the pair, issued by the leader: A rows 0-127 and B rows 0..N/2-1
// from the leader's shared memory, the rest from the peer's at the same offsets;
// D rows 0-127 into the leader's TMEM, 128-255 into the peer's
__device__ __forceinline__ void mma_issue_pair(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtm),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// arrive on the barrier at this offset in both CTAs once the pair's MMAs issued
// so far are complete
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile that TMA wrote with the
// configuration's swizzle: 8-row atoms SBO bytes apart, descriptor version 1,
// swizzle layout code at bits 61-63.
template <int KC>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(KCfg<KC>::SBO >> 4) << 32) |
           ((uint64_t)1 << 46) | (KCfg<KC>::LAYOUT << 61);
}

template <bool TF32>
__device__ __forceinline__ void mma_issue(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 16 consecutive FP32 columns: thread = lane, v[c] = column col + c.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"r"(EPI_THREADS) : "memory"); }

__device__ __forceinline__ void split_store(__nv_bfloat16* hi, __nv_bfloat16* lo, int64_t off, float v, bool with_lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[off] = h;
    if (with_lo) lo[off] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// v rounded to TF32 (10 explicit mantissa bits, nearest, ties away), in FP32.
__device__ __forceinline__ float to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// Operand image entry `off` of value v: BF16 hi (+ lo) or, in the TF32 and FP32
// modes, TF32 values in FP32 containers (the storage of `hi` and `lo` then holds
// floats): hi = tf32(v) and, where a lo image exists, lo = tf32(v - hi).
__device__ __forceinline__ void image_store(__nv_bfloat16* hi, __nv_bfloat16* lo, int64_t off, float v, bool with_lo,
                                            bool tf32) {
    if (tf32) {
        const float h = to_tf32(v);
        reinterpret_cast<float*>(hi)[off] = h;
        if (with_lo && lo) reinterpret_cast<float*>(lo)[off] = to_tf32(v - h);
    } else {
        split_store(hi, lo, off, v, with_lo);
    }
}

struct TcMaps {
    CUtensorMap a0, a1, b0, b1;   // a0/a1: hi/lo of W or L; b0/b1: hi/lo of the B operand
};

struct TcArgs {
    int64_t N, M, ldk, n_rt, n_vec;   // n_vec: B rows (2M, or K vectors in the field mode)
    float hdtG, hdtw, sgdt, sdt;      // dt G / 2, dt w / 2 (w: scale of the W image), sqrt(G dt), sqrt(w dt)
    float fsc;                        // FIELD: factor applied to the accumulator (the image's scale)
    int renorm;
    int integ;                        // TWA_INT_HEUN or TWA_INT_MIDPOINT
    int band;                         // one-product W tiles: see two_product_stages
    const float *X, *Y, *Z;           // PRED: s; CORR: s~ (midpoint scheme: s)
    const float *X0, *Y0, *Z0;        // CORR: s, the state before the step
    const float *Bnx, *Bny;           // PRED, CORR: noise part of the field increment
    float *oX, *oY, *oZ;              // PRED: s~ (not written by the midpoint scheme); CORR: s'
    float *oBnx, *oBny;               // LETA
    __nv_bfloat16 *oHi, *oLo;         // images of the output state (midpoint scheme's
                                      // predictor: of the midpoint (s + s~)/2)
    const float* XI;                  // LETA: collective normals [M][2]
    const float* part_in;             // sums of the input state, [n_rt][M][4]
    float* part_out;                  // sums of the output state
    float* field_out;                 // FIELD: [n_vec][N]
    unsigned long long* flags;
    // launch argument of the dense step's MIX launches: the noise of step
    // *nz_dt + nz_toff (BF16 images of eta into nz_E0 / nz_E1 and xi into
    // nz_XI0 / nz_XI1 by the parity of that step), draws [nz_lo, nz_hi) of the
    // M x (N + 1) in the order of k_noise_tc, drawn by the epilogue threads
    // between tiles (nz_E0 = NULL: none)
    __nv_bfloat16 *nz_E0, *nz_E1;
    float *nz_XI0, *nz_XI1;
    const int64_t* nz_dt;
    int64_t nz_toff, nz_lo, nz_hi, nz_m0;
    uint64_t nz_seed;
};

// A batch of problems in one launch: descriptor table (tensor maps in global
// memory, 64-byte aligned) and the prefix sums of their tile counts.
struct GroupDesc {   // 64-byte aligned through its tensor maps
    TcMaps maps;
    TcArgs args;
    int mode;               // kernel mode of this problem's tiles (MODE_MIX launches)
    int nterms;             // tensor-core products per entry of this problem's tiles
};
struct Group {
    const GroupDesc* desc;
    const int64_t* start;   // [count + 1]: first flat tile of each problem
    int count;              // 0: a single problem, given by the launch arguments
    // optional explicit schedule: CTA b runs flat tiles sched[sched_start[b] ..
    // sched_start[b + 1]) in that order (else tiles b, b + grid, b + 2 grid, ...)
    const int32_t* sched = nullptr;
    const int32_t* sched_start = nullptr;
    int ctas = 0;   // grid of a scheduled launch
};

// K stages [kb0, kb1) of a tile of row unit rt (MROWS rows) that take two
// products although the tile's product count is one (W in BF16L2, W and L in
// BF16B): the entries
// with j in [u - 64 band, u + 256 + 64 band), u = the 256-row-aligned start of
// the tile's rows, i.e. every entry within 64 band columns of the diagonal (and
// the same set of entries on single CTAs and on CTA pairs, whatever the K-stage
// width bk, a divisor of 64). Off this band W is one BF16 product.
__host__ __device__ __forceinline__ void two_product_stages(int64_t rt, int mrows, int bk, int band, int& kb0,
                                                            int& kb1) {
    const int64_t u = rt * mrows / 256 * 256;
    kb0 = (int)((u - 64 * (int64_t)band) / bk);
    kb1 = (int)((u + 256 + 64 * (int64_t)band) / bk);
}

// PAIR: launched in clusters of two CTAs that share each 256-row tile (row tiles
// 2r and 2r + 1 of row unit r): both stream their own A rows and half of the B
// rows, the leader (rank 0) issues the cta_group::2 MMAs, and each runs the
// epilogue of its own 128 rows from its own TMEM.
template <int MODE, int NT, int BN, int KC, bool PAIR = false>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc(const __grid_constant__ TcMaps maps, const TcArgs args,
                                                   const Group grp) {
    using G_ = Geo<BN, KC, PAIR>;
    static_assert(!(PAIR && KCfg<KC>::TF32), "CTA pairs run the BF16 configurations");
    constexpr int BK = G_::BK, STAGES = G_::STAGES, NTRAJ = G_::NTRAJ;
    constexpr bool TFM = KCfg<KC>::TF32;   // TF32 mode: kind::tf32 MMAs, FP32-container images
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* tiles = smem;
    uint64_t* full = (uint64_t*)(smem + G_::TILES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;            // [2] accumulator ready
    uint64_t* tempty = tfull + 2;                // [2] accumulator drained by the epilogue
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    float* sS = (float*)(tmem_slot + 4);         // [NTRAJ][2] input sums (or xi) of the tile's trajectories
    float* red = sS + 2 * NTRAJ * 2;             // [4][NTRAJ][3]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // scheduling unit: the CTA, or the cluster of a pair (both CTAs walk its list)
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const int64_t unit = PAIR ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;
    const int64_t units = PAIR ? (int64_t)(gridDim.x >> 1) : (int64_t)gridDim.x;
    // row tiles are handed out in row units: one 128-row tile, or two for a pair
    auto row_units = [](int64_t n_rt) -> int64_t { return PAIR ? (n_rt + 1) >> 1 : n_rt; };
    // flat tile list: one problem, or the problems of the group one after another
    const int64_t ntiles = grp.count ? grp.start[grp.count] : row_units(args.n_rt) * ((args.n_vec + BN - 1) / BN);
    // this unit's tiles: the k-th is tile_of(k), k < n_mine
    const int64_t n_mine = grp.sched ? (int64_t)(grp.sched_start[unit + 1] - grp.sched_start[unit])
                                     : (unit < ntiles ? (ntiles - 1 - unit) / units + 1 : 0);
    auto tile_of = [&](int64_t k) -> int64_t {
        return grp.sched ? (int64_t)grp.sched[grp.sched_start[unit] + k] : unit + k * units;
    };
    // problem of flat tile t, the tile's (row tile, trajectory tile) within it, and
    // its mode and term count (the template's, except in MODE_MIX launches)
    auto resolve = [&](int64_t t, const TcMaps*& mp, const TcArgs*& ap, int64_t& rt, int64_t& ct, int& md,
                       int& nt) {
        int64_t tl = t;
        md = MODE;
        nt = NT;
        if (grp.count == 0) {
            mp = &maps;
            ap = &args;
        } else {
            int lo = 0, hi = grp.count - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (grp.start[mid] <= t) lo = mid;
                else hi = mid - 1;
            }
            mp = &grp.desc[lo].maps;
            ap = &grp.desc[lo].args;
            tl = t - grp.start[lo];
            if (MODE == MODE_MIX) {
                // each problem's mode and product count from its descriptor: W.s
                // tiles take the precision's W count (the template's), L.eta tiles
                // that of L (two products when L is split and the noise operand is
                // a single BF16 value; three in the FP32 mode, whose eta is split too)
                md = grp.desc[lo].mode;
                nt = grp.desc[lo].nterms;
            }
        }
        const int64_t nct = (ap->n_vec + BN - 1) / BN;
        rt = tl / nct;
        ct = tl - rt * nct;
        // L.eta: row unit r needs (r + 1) M-rows of K (triangular L); hand out the
        // longest tiles first so the persistent CTAs finish together
        if (md == MODE_LETA) rt = row_units(ap->n_rt) - 1 - rt;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            // a pair's accumulator is free once the epilogues of both CTAs drained it
            mbar_init(&tempty[b], PAIR ? 2 * EPI_WARPS : EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        // a pair allocates collectively: the same columns in both CTAs' TMEM
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(G_::NCOLS));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(G_::NCOLS));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();   // both CTAs' barriers initialised before any cross-CTA arrival
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto k_tiles = [&](const TcArgs* ap, int64_t rt, int md) -> int {
        const int nk = (int)((ap->N + BK - 1) / BK);
        if (md != MODE_LETA) return nk;
        const int k1 = (int)(((rt + 1) * G_::MROWS + BK - 1) / BK);   // L is lower triangular (rt: row unit)
        return k1 < nk ? k1 : nk;
    };

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            uint32_t stage = 0, ph = 0;
            int last_ph[STAGES];
            bool issued[STAGES];
            for (int s = 0; s < STAGES; ++s) {
                issued[s] = false;
                last_ph[s] = 0;
            }
            bool ok = true;
            const TcMaps* prev = nullptr;
            for (int64_t k = 0; k < n_mine && ok; ++k) {
                const int64_t t = tile_of(k);
                const TcMaps* mp;
                const TcArgs* ap;
                int64_t rt, ct;
                int md, nt;
                resolve(t, mp, ap, rt, ct, md, nt);
                // operands of this tile: W/L hi (+ lo), B hi (+ lo; never in a
                // one-B configuration, which the host uses for at most two products);
                // a one-product W tile takes the lo image on its band stages
                const int nb = (nt == 3 && !KCfg<KC>::ONE_B) ? 2 : 1;
                int kb0 = 0, kb1 = 0;
                if (nt == 1 && ap->band > 0) two_product_stages(rt, G_::MROWS, BK, ap->band, kb0, kb1);
                if (grp.count && mp != prev) {
                    // descriptors written to global memory before the launch: make them
                    // visible to the tensor-map proxy before the first copy through them
                    const CUtensorMap* ms[4] = {&mp->a0, &mp->a1, &mp->b0, &mp->b1};
                    for (int k = 0; k < 4; ++k)
                        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(ms[k]) : "memory");
                    prev = mp;
                }
                // a pair's CTA: its own row tile of the unit, its half of the B rows
                const int y_a = (int)((PAIR ? 2 * rt + rank : rt) * BM);
                const int y_b = (int)(ct * BN + (PAIR ? rank * (BN / 2) : 0));
                const int nkt = k_tiles(ap, rt, md);
                for (int kt = 0; kt < nkt; ++kt) {
                    if (!mbar_wait(&empty[stage], ph ^ 1u, args.flags, true)) {
                        ok = false;
                        break;
                    }
                    const int na = (nt >= 2 || (kt >= kb0 && kt < kb1)) ? 2 : 1;
                    const uint32_t tx = na * G_::A_BYTES + nb * G_::B_BYTES;
                    uint8_t* st = tiles + stage * G_::STAGE_BYTES;
                    const int kx = kt * BK;
                    if constexpr (PAIR) {
                        // both CTAs' copies complete on the leader's barrier, which
                        // expects the bytes of the two
                        if (rank == 0) mbar_expect_tx(&full[stage], 2 * tx);
                        const uint32_t fb = cluster_addr(&full[stage], 0);
                        tma_load_pair(st, &mp->a0, fb, kx, y_a);
                        if (na == 2) tma_load_pair(st + G_::A_BYTES, &mp->a1, fb, kx, y_a);
                        tma_load_pair(st + 2 * G_::A_BYTES, &mp->b0, fb, kx, y_b);
                        if (nb == 2) tma_load_pair(st + 2 * G_::A_BYTES + G_::B_BYTES, &mp->b1, fb, kx, y_b);
                    } else {
                        mbar_expect_tx(&full[stage], tx);
                        tma_load(st, &mp->a0, &full[stage], kx, y_a);
                        if (na == 2) tma_load(st + G_::A_BYTES, &mp->a1, &full[stage], kx, y_a);
                        tma_load(st + 2 * G_::A_BYTES, &mp->b0, &full[stage], kx, y_b);
                        if (nb == 2) tma_load(st + 2 * G_::A_BYTES + G_::B_BYTES, &mp->b1, &full[stage], kx, y_b);
                    }
                    issued[stage] = true;
                    last_ph[stage] = (int)ph;
                    if (++stage == STAGES) {
                        stage = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                // let copies already in flight land before the CTA can exit
                if (PAIR && rank == 1) {
                    // they complete on the leader's barriers, which this CTA cannot
                    // wait on: give them a bounded time (a copy takes microseconds)
                    const uint64_t t0 = gtimer();
                    while (gtimer() - t0 < 200000ull) {
                    }
                } else {
                    for (int s = 0; s < STAGES; ++s)
                        if (issued[s]) mbar_wait(&full[s], (uint32_t)last_ph[s], args.flags, false);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (a pair's leader only) ----------------
        // one MMA: this CTA's (cta_group::1), or the pair's 256-row one
        auto issue = [&](uint32_t dcol, uint64_t ad, uint64_t bd, uint32_t acc) {
            if constexpr (PAIR) mma_issue_pair(dcol, ad, bd, G_::IDESC, acc);
            else mma_issue<TFM>(dcol, ad, bd, G_::IDESC, acc);
        };
        auto commit = [&](uint64_t* bar) {
            if constexpr (PAIR) mma_commit_pair(bar);   // both CTAs' barriers
            else mma_commit(bar);
        };
        if (lane == 0 && (!PAIR || rank == 0)) {
            uint32_t stage = 0, ph = 0;
            bool ok = true;
            int it = 0, last_b = -1;
            uint32_t last_par = 0;
            for (int64_t k = 0; k < n_mine && ok; ++k, ++it) {
                const int64_t t = tile_of(k);
                const int b = it & 1;
                const uint32_t use = (uint32_t)(it >> 1);
                if (!mbar_wait<PAIR>(&tempty[b], (use & 1u) ^ 1u, args.flags, true)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dcol = tmem + (uint32_t)(b * BN);
                const TcMaps* mp;
                const TcArgs* ap;
                int64_t rt, ct;
                int md, nt;
                resolve(t, mp, ap, rt, ct, md, nt);
                const int nkt = k_tiles(ap, rt, md);
                int kb0 = 0, kb1 = 0;
                if (nt == 1 && ap->band > 0) two_product_stages(rt, G_::MROWS, BK, ap->band, kb0, kb1);
                for (int kt = 0; kt < nkt; ++kt) {
                    if (!mbar_wait(&full[stage], ph, args.flags, true)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const bool lo_a = nt == 2 || (kt >= kb0 && kt < kb1);   // A lo against B hi
                    const uint32_t a0 = smem_u32(tiles + stage * G_::STAGE_BYTES);
                    const uint32_t a1 = a0 + G_::A_BYTES, b0 = a0 + 2 * G_::A_BYTES, b1 = b0 + G_::B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < G_::MMAS; ++kk) {
                        const uint32_t ko = kk * 32;   // 16 BF16 or 8 TF32 = 32 B along the swizzled row
                        issue(dcol, sdesc<KC>(a0 + ko), sdesc<KC>(b0 + ko), (kt > 0 || kk > 0) ? 1u : 0u);
                        if (nt == 3 && !KCfg<KC>::ONE_B) {
                            issue(dcol, sdesc<KC>(a0 + ko), sdesc<KC>(b1 + ko), 1u);
                            issue(dcol, sdesc<KC>(a1 + ko), sdesc<KC>(b0 + ko), 1u);
                        }
                        if (lo_a) issue(dcol, sdesc<KC>(a1 + ko), sdesc<KC>(b0 + ko), 1u);
                    }
                    commit(&empty[stage]);
                    if (++stage == STAGES) {
                        stage = 0;
                        ph ^= 1u;
                    }
                }
                commit(&tfull[b]);   // this tile's accumulator is complete (or drained, after an abort)
                last_b = b;
                last_par = use & 1u;
            }
            // MMAs still in flight must finish before the accumulators are freed
            if (last_b >= 0) mbar_wait(&tfull[last_b], last_par, args.flags, false);
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int q = warp & 3;              // TMEM lane quadrant of this warp
        const int grp_e = (warp - 2) >> 2;   // which share of the accumulator columns
        const int et = threadIdx.x - 64;     // 0 .. EPI_THREADS - 1
        // MIX launches of the dense step: this CTA's share of the noise draws of a
        // later step, in `parts` pieces, one after each of its tiles (all of it
        // at the end when the CTA has no tile)
        const TcArgs& la = args;
        auto draw_noise = [&](int64_t part, int64_t parts) {
            const int64_t per = (la.nz_hi - la.nz_lo + gridDim.x - 1) / gridDim.x;
            const int64_t c0 = la.nz_lo + (int64_t)blockIdx.x * per;
            const int64_t c1 = c0 + per < la.nz_hi ? c0 + per : la.nz_hi;
            const int64_t sub = (per + parts - 1) / parts;
            const int64_t s0 = c0 + part * sub;
            const int64_t s1 = s0 + sub < c1 ? s0 + sub : c1;
            if (s0 >= s1) return;
            const int64_t NP = la.N + 1;
            const int64_t st = *la.nz_dt + la.nz_toff;
            __nv_bfloat16* E = (st & 1) ? la.nz_E1 : la.nz_E0;
            float* XI = (st & 1) ? la.nz_XI1 : la.nz_XI0;
            for (int64_t e = s0 + et; e < s1; e += EPI_THREADS) {
                const int64_t m = e / NP, i = e - m * NP;
                float gx, gy;
                normal2_f32(la.nz_seed, (uint32_t)(la.nz_m0 + m), (uint32_t)st, (uint32_t)i, gx, gy);
                if (i < la.N) {
                    E[(2 * m) * la.ldk + i] = __float2bfloat16_rn(gx);
                    E[(2 * m + 1) * la.ldk + i] = __float2bfloat16_rn(gy);
                } else {
                    XI[2 * m] = gx;
                    XI[2 * m + 1] = gy;
                }
            }
        };
        const bool nz = MODE == MODE_MIX && la.nz_E0 != nullptr;
        if (nz && n_mine == 0) draw_noise(0, 1);
        int it = 0;
        for (int64_t k = 0; k < n_mine; ++k, ++it) {
            const int64_t t = tile_of(k);
            const int b = it & 1;
            const uint32_t use = (uint32_t)(it >> 1);
            const TcMaps* mp_;
            const TcArgs* ap_;
            int64_t rt, ct;
            int md, nt;
            resolve(t, mp_, ap_, rt, ct, md, nt);
            if constexpr (PAIR) rt = 2 * rt + rank;   // this CTA's row tile of the unit
            const TcArgs& args = *ap_;        // this tile's problem (shadows the launch argument)
            const int64_t M = args.M;
            const float hdtG = args.hdtG, hdtw = args.hdtw, sdt = args.sdt, sgdt = args.sgdt, fsc = args.fsc;
            // every rounding of the epilogue is spelled out (fmaf, __fmul_rn,
            // __fadd_rn), so that all kernel variants give the same bits
            const int64_t i0 = rt * BM, n0 = ct * BN, m0 = n0 >> 1;
            const int64_t i = i0 + 32 * q + lane;        // site of this thread
            const bool site_ok = i < args.N;
            epi_sync();                                   // smem of the previous tile is free
            if (md == MODE_PRED || md == MODE_CORR) {
                for (int j = et; j < NTRAJ; j += EPI_THREADS) {
                    const int64_t m = m0 + j;
                    float sx = 0.f, sy = 0.f;
                    if (m < M) {
                        for (int64_t r = 0; r < args.n_rt; ++r) {
                            const float4 v = *(const float4*)(args.part_in + (r * M + m) * 4);
                            sx += v.x;
                            sy += v.y;
                        }
                    }
                    sS[2 * j] = sx;
                    sS[2 * j + 1] = sy;
                }
            } else if (md == MODE_LETA) {
                for (int j = et; j < NTRAJ; j += EPI_THREADS) {
                    const int64_t m = m0 + j;
                    sS[2 * j] = (m < M) ? args.XI[2 * m] : 0.f;
                    sS[2 * j + 1] = (m < M) ? args.XI[2 * m + 1] : 0.f;
                }
            }
            epi_sync();
            const bool acc_ok = mbar_wait(&tfull[b], use & 1u, args.flags, true);
            tc_fence_after();
            // warp-uniform, so that the .sync.aligned TMEM loads and the shuffles
            // below are reached by every lane or by none
            const bool live =
                __all_sync(0xffffffffu, acc_ok && (((volatile unsigned long long*)args.flags)[FLAG_TIMEOUT] == 0ull));
            const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN);
            unsigned nonfinite = 0;
            // the accumulator pass, compiled once per epilogue mode EM, so that each
            // mode's loop is scheduled as in a kernel of that mode alone
            auto run_tile = [&](auto em_tag) {
                constexpr int EM = decltype(em_tag)::value;
                constexpr bool WITH_LO = (NT == 3);   // images of the W.s operand: hi + lo
                for (int c = grp_e * (BN / 16) / EPI_GROUPS; c < (grp_e + 1) * (BN / 16) / EPI_GROUPS; ++c) {
                    float pv[16];
                    tmem_ld16(trow + 16 * c, pv);
                    tmem_ld_wait();
                    if constexpr (EM == MODE_FIELD) {
                        if (site_ok) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const int64_t n = n0 + 16 * c + j;
                                if (n < args.n_vec) args.field_out[n * args.N + i] = __fmul_rn(fsc, pv[j]);
                            }
                        }
                    } else if constexpr (EM == MODE_LETA) {
                        // noise part of the field increment: sqrt(G dt) xi^a - sqrt(dt) (L eta^a)_i,
                        // sqrt(dt) L = sqrt(w dt) times the accumulated image of L / sqrt(w)
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int jl = 8 * c + jj;
                            const int64_t m = m0 + jl;
                            if (!site_ok || m >= M) continue;
                            const int64_t e = m * args.N + i;
                            args.oBnx[e] = fmaf(-sdt, pv[2 * jj], __fmul_rn(sgdt, sS[2 * jl]));
                            args.oBny[e] = fmaf(-sdt, pv[2 * jj + 1], __fmul_rn(sgdt, sS[2 * jl + 1]));
                        }
                    } else {
                        float rx[8], ry[8], rz[8];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int jl = 8 * c + jj;            // local trajectory
                            const int64_t m = m0 + jl;
                            rx[jj] = ry[jj] = rz[jj] = 0.f;
                            if (!site_ok || m >= M) continue;
                            const int64_t e = m * args.N + i;
                            const float x = args.X[e], y = args.Y[e], z = args.Z[e];
                            // B^a = 1/2 (G S^a - P^a) dt + noise part, P = w times the
                            // accumulated product of the image of W / w
                            const float Bxv = fmaf(-hdtw, pv[2 * jj], fmaf(hdtG, sS[2 * jl], args.Bnx[e]));
                            const float Byv = fmaf(-hdtw, pv[2 * jj + 1], fmaf(hdtG, sS[2 * jl + 1], args.Bny[e]));
                            const int64_t r0 = (2 * m) * args.ldk + i;
                            if constexpr (EM == MODE_PRED) {
                                float xp, yp, zp;
                                if (args.integ == TWA_INT_MIDPOINT) {
                                    // the corrector's field point (s + s~)/2; only its
                                    // images and sums are needed
                                    mid_rotation_f32(x, y, z, Bxv, Byv, xp, yp, zp);
                                } else {
                                    // f = s x (B^y, -B^x, 0); s~ = s + f
                                    const float fx = __fmul_rn(z, Bxv), fy = __fmul_rn(z, Byv);
                                    const float fz = -fmaf(x, Bxv, __fmul_rn(y, Byv));
                                    xp = __fadd_rn(x, fx);
                                    yp = __fadd_rn(y, fy);
                                    zp = __fadd_rn(z, fz);
                                    args.oX[e] = xp;
                                    args.oY[e] = yp;
                                    args.oZ[e] = zp;
                                }
                                image_store(args.oHi, args.oLo, r0, xp, WITH_LO, TFM);
                                image_store(args.oHi, args.oLo, r0 + args.ldk, yp, WITH_LO, TFM);
                                rx[jj] = xp;
                                ry[jj] = yp;
                                rz[jj] = zp;
                            } else {
                                float nx, ny, nz;
                                if (args.integ == TWA_INT_MIDPOINT) {
                                    // (x, y, z) = s; field of the midpoint state:
                                    // s' = 2 m - s of the rotation from s
                                    float mx, my, mz;
                                    mid_rotation_f32(x, y, z, Bxv, Byv, mx, my, mz);
                                    nx = fmaf(2.0f, mx, -x);
                                    ny = fmaf(2.0f, my, -y);
                                    nz = fmaf(2.0f, mz, -z);
                                } else {
                                    // corrector: s' = s + (f(s) + f(s~))/2 = (s + s~)/2 + f(s~)/2,
                                    // then |s'| = sqrt(3)
                                    const float hx = __fmul_rn(0.5f, __fadd_rn(args.X0[e], x));
                                    const float hy = __fmul_rn(0.5f, __fadd_rn(args.Y0[e], y));
                                    const float hz = __fmul_rn(0.5f, __fadd_rn(args.Z0[e], z));
                                    nx = fmaf(0.5f, __fmul_rn(z, Bxv), hx);
                                    ny = fmaf(0.5f, __fmul_rn(z, Byv), hy);
                                    nz = fmaf(-0.5f, fmaf(x, Bxv, __fmul_rn(y, Byv)), hz);
                                }
                                if (args.renorm) {
                                    const float s = sqrtf(3.0f / fmaf(nx, nx, fmaf(ny, ny, __fmul_rn(nz, nz))));
                                    nx = __fmul_rn(nx, s);
                                    ny = __fmul_rn(ny, s);
                                    nz = __fmul_rn(nz, s);
                                }
                                if (!(isfinite(nx) && isfinite(ny) && isfinite(nz))) ++nonfinite;
                                args.oX[e] = nx;
                                args.oY[e] = ny;
                                args.oZ[e] = nz;
                                image_store(args.oHi, args.oLo, r0, nx, WITH_LO, TFM);
                                image_store(args.oHi, args.oLo, r0 + args.ldk, ny, WITH_LO, TFM);
                                rx[jj] = nx;
                                ry[jj] = ny;
                                rz[jj] = nz;
                            }
                        }
                        // partial sums over this warp's 32 sites
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
#pragma unroll
                            for (int o = 16; o; o >>= 1) {
                                rx[jj] += __shfl_xor_sync(0xffffffffu, rx[jj], o);
                                ry[jj] += __shfl_xor_sync(0xffffffffu, ry[jj], o);
                                rz[jj] += __shfl_xor_sync(0xffffffffu, rz[jj], o);
                            }
                        }
                        if (lane == 0) {
#pragma unroll
                            for (int jj = 0; jj < 8; ++jj) {
                                float* rr = red + (q * NTRAJ + 8 * c + jj) * 3;
                                rr[0] = rx[jj];
                                rr[1] = ry[jj];
                                rr[2] = rz[jj];
                            }
                        }
                    }
                }
            };
            if (live) {
                if constexpr (MODE != MODE_MIX) {
                    run_tile(std::integral_constant<int, MODE>{});
                } else {
                    if (md == MODE_CORR) run_tile(std::integral_constant<int, MODE_CORR>{});
                    else if (md == MODE_PRED) run_tile(std::integral_constant<int, MODE_PRED>{});
                    else run_tile(std::integral_constant<int, MODE_LETA>{});
                }
            }
            // accumulator b may be overwritten by the next tile's MMAs
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR && rank == 1) mbar_arrive_cluster(cluster_addr(&tempty[b], 0));   // the leader's
                else mbar_arrive(&tempty[b]);
            }
            if (md == MODE_CORR) {
                const unsigned tot = __reduce_add_sync(0xffffffffu, nonfinite);
                if (lane == 0 && tot) atomicAdd(&args.flags[FLAG_NONFINITE], (unsigned long long)tot);
            }
            // (md is the same for the four epilogue warps: they walk the same tiles)
            if (md == MODE_PRED || md == MODE_CORR) {
                epi_sync();   // every epilogue thread, live or not
                for (int j = et; j < NTRAJ; j += EPI_THREADS) {
                    const int64_t m = m0 + j;
                    // (a pair's second row tile may lie past the last one)
                    if (!live || m >= M || rt >= args.n_rt) continue;
                    float4 o;
                    o.x = red[(0 * NTRAJ + j) * 3] + red[(1 * NTRAJ + j) * 3] + red[(2 * NTRAJ + j) * 3] +
                          red[(3 * NTRAJ + j) * 3];
                    o.y = red[(0 * NTRAJ + j) * 3 + 1] + red[(1 * NTRAJ + j) * 3 + 1] + red[(2 * NTRAJ + j) * 3 + 1] +
                          red[(3 * NTRAJ + j) * 3 + 1];
                    o.z = red[(0 * NTRAJ + j) * 3 + 2] + red[(1 * NTRAJ + j) * 3 + 2] + red[(2 * NTRAJ + j) * 3 + 2] +
                          red[(3 * NTRAJ + j) * 3 + 2];
                    o.w = 0.f;
                    *(float4*)(args.part_out + (rt * M + m) * 4) = o;
                }
            }
            if (nz) draw_noise(k, n_mine);
        }
    }
    __syncthreads();
    // no CTA of a pair leaves while the other may still reach its shared memory
    if constexpr (PAIR) cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G_::NCOLS));
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G_::NCOLS));
    }
}

// ---------------------------------------------------------------------------
// elementwise kernels of the mixed path

// One bounded wait, by the routine every tensor-core kernel uses on its
// mbarriers, on a barrier that nothing arrives on: it gives up after limit_ns
// and counts the timeout in flags[FLAG_TIMEOUT], touching nothing else.
__global__ void k_wait_probe(unsigned long long* flags, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_wait(&bar, 0u, flags, false, limit_ns);
    }
}

// Images of inv * src (inv: the reciprocal of the scale the epilogue applies).
__global__ void k_split_matrix(const double* src, int64_t N, int64_t ldk, __nv_bfloat16* hi, __nv_bfloat16* lo,
                               int tf32, double inv) {
    const int64_t n2 = N * ldk;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / ldk, k = e - r * ldk;
        const float v = (k < N) ? (float)(inv * src[r * N + k]) : 0.f;
        if (tf32) {   // TF32 images in FP32 containers: hi, and lo where it exists
            const float h = to_tf32(v);
            reinterpret_cast<float*>(hi)[e] = h;
            if (lo) reinterpret_cast<float*>(lo)[e] = to_tf32(v - h);
            continue;
        }
        // hi = bf16(v), lo = bf16(v - hi): the pair carries ~16 significant bits
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[e] = h;
        lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

__global__ void k_init_tc(float* X, float* Y, float* Z, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t M, int64_t N,
                          int64_t ldk, uint64_t seed, float init_sz, int64_t m0, int tf32) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N;
    double sx, sy;
    init_signs(seed, (uint32_t)(m0 + m), (uint32_t)i, sx, sy);
    X[e] = (float)sx;
    Y[e] = (float)sy;
    Z[e] = init_sz;
    if (tf32) {   // +-1 is exact in TF32
        reinterpret_cast<float*>(hi)[(2 * m) * ldk + i] = (float)sx;
        reinterpret_cast<float*>(hi)[(2 * m + 1) * ldk + i] = (float)sy;
        if (lo) {
            reinterpret_cast<float*>(lo)[(2 * m) * ldk + i] = 0.f;
            reinterpret_cast<float*>(lo)[(2 * m + 1) * ldk + i] = 0.f;
        }
        return;
    }
    hi[(2 * m) * ldk + i] = __float2bfloat16_rn((float)sx);
    hi[(2 * m + 1) * ldk + i] = __float2bfloat16_rn((float)sy);
    lo[(2 * m) * ldk + i] = __float2bfloat16_rn(0.f);
    lo[(2 * m + 1) * ldk + i] = __float2bfloat16_rn(0.f);
}

// Images of an arbitrary FP32 state (after set_state).
__global__ void k_images_tc(const float* X, const float* Y, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t M,
                            int64_t N, int64_t ldk, int tf32) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t m = e / N, i = e - m * N;
    image_store(hi, lo, (2 * m) * ldk + i, X[e], true, tf32);
    image_store(hi, lo, (2 * m + 1) * ldk + i, Y[e], true, tf32);
}

// part[r][m] = sums over sites [128 r, 128 r + 128) of (x, y, z); one warp per (r, m).
__global__ void k_part_tc(const float* X, const float* Y, const float* Z, float* part, int64_t M, int64_t N,
                          int64_t n_rt) {
    const int64_t w = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (w >= n_rt * M) return;
    const int64_t r = w / M, m = w - r * M;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int k = lane; k < BM; k += 32) {
        const int64_t i = r * BM + k;
        if (i < N) {
            sx += X[m * N + i];
            sy += Y[m * N + i];
            sz += Z[m * N + i];
        }
    }
    for (int o = 16; o; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    if (lane == 0) *(float4*)(part + (r * M + m) * 4) = make_float4(sx, sy, sz, 0.f);
}

// Noise of step t = *d_t + toff: eta (FP32 Box-Muller, rounded to BF16, or to TF32
// in an FP32 container, with a TF32 lo image Elo in the FP32 mode) into the
// B-operand image rows 2m / 2m+1, and the collective pair xi (site index N) into XI.
// Noise of step s = *d_t + toff (pump normals as the B-operand image, collective
// normals into XI) into the buffers of s's parity: (E0, Elo0, XI0) for even s,
// (E1, Elo1, XI1) for odd s (the same pointers twice where one buffer serves).
__global__ void k_noise_tc(__nv_bfloat16* E0, __nv_bfloat16* Elo0, float* XI0, __nv_bfloat16* E1,
                           __nv_bfloat16* Elo1, float* XI1, int64_t M, int64_t N, int64_t ldk, uint64_t seed,
                           const int64_t* d_t, int64_t toff, int64_t m0, int tf32) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t NP = N + 1;
    if (e >= M * NP) return;
    const int64_t m = e / NP, i = e - m * NP;
    const int64_t s = *d_t + toff;
    const uint32_t t = (uint32_t)s;
    __nv_bfloat16* E = (s & 1) ? E1 : E0;
    __nv_bfloat16* Elo = (s & 1) ? Elo1 : Elo0;
    float* XI = (s & 1) ? XI1 : XI0;
    float gx, gy;
    normal2_f32(seed, (uint32_t)(m0 + m), t, (uint32_t)i, gx, gy);
    if (i < N) {
        image_store(E, Elo, (2 * m) * ldk + i, gx, Elo != nullptr, tf32);
        image_store(E, Elo, (2 * m + 1) * ldk + i, gy, Elo != nullptr, tf32);
    } else {
        XI[2 * m] = gx;
        XI[2 * m + 1] = gy;
    }
}

// S^a of trajectory m in FP64 from the per-row-tile partial sums, one warp per
// trajectory: lane l adds tiles l, l + 32, ... in order, then a butterfly over
// the lanes (a fixed order, so every run gives the same bits). All lanes
// receive the sums.
__device__ __forceinline__ void warp_tile_sums(const float* part, int64_t M, int64_t n_rt, int64_t m, int lane,
                                               double& sx, double& sy, double& sz) {
    sx = sy = sz = 0.0;
    for (int64_t r = lane; r < n_rt; r += 32) {
        const float4 v = *(const float4*)(part + (r * M + m) * 4);
        sx += v.x;
        sy += v.y;
        sz += v.z;
    }
    for (int o = 16; o; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
}

// Window moments S^z, A, A^2, A S^z, (S^z)^2 of one trajectory (A = |S^x + i S^y|^2 / 4).
__device__ __forceinline__ void add_moments(double* mm, double sx, double sy, double sz) {
    const double A = 0.25 * (sx * sx + sy * sy);
    mm[0] += sz;
    mm[1] += A;
    mm[2] += A * A;
    mm[3] += A * sz;
    mm[4] += sz * sz;
}

// Closing kernel: S^a from the corrector's partial sums (one warp per
// trajectory), the FP64 window moments, and the step counter (last block).
__global__ void k_close_tc(const float* part, int64_t M, int64_t n_rt, double* mom, int64_t* d_t, int64_t n_window,
                           int64_t n_stride, int64_t* d_count, unsigned long long* flags) {
    const int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t t1 = *d_t + 1;
    const bool sample = window_sample(t1, n_window, n_stride);
    if (m < M && sample) {   // warp-uniform
        double sx, sy, sz;
        warp_tile_sums(part, M, n_rt, m, lane, sx, sy, sz);
        if (lane == 0) add_moments(mom + 5 * m, sx, sy, sz);
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

// ---------------------------------------------------------------------------
// grouped per-step kernels of a batch of problems

struct StepDesc {
    __nv_bfloat16 *E, *E1;   // noise images of even / odd steps
    float *XI, *XI1;
    const float* part;
    double* mom;
    int64_t* d_t;
    int64_t* d_count;
    int64_t M, N, ldk, n_rt, n_window, n_stride, m0;
    uint64_t seed;
};

__device__ __forceinline__ int find_problem(const int64_t* start, int n, int64_t e) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Noise of every problem's step *d_t + toff (start = prefix of M (N + 1)), into
// the buffers of that step's parity.
__global__ void k_noise_group(const StepDesc* sd, const int64_t* start, int n, int64_t toff) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= start[n]) return;
    const int p = find_problem(start, n, e);
    const StepDesc& d = sd[p];
    const int64_t el = e - start[p], NP = d.N + 1;
    const int64_t m = el / NP, i = el - m * NP;
    float gx, gy;
    const int64_t st = *d.d_t + toff;
    normal2_f32(d.seed, (uint32_t)(d.m0 + m), (uint32_t)st, (uint32_t)i, gx, gy);
    __nv_bfloat16* E = (st & 1) ? d.E1 : d.E;
    float* XI = (st & 1) ? d.XI1 : d.XI;
    if (i < d.N) {
        E[(2 * m) * d.ldk + i] = __float2bfloat16_rn(gx);
        E[(2 * m + 1) * d.ldk + i] = __float2bfloat16_rn(gy);
    } else {
        XI[2 * m] = gx;
        XI[2 * m + 1] = gy;
    }
}

// Window moments of every problem (start = prefix of M); counters advance later.
__global__ void k_close_group(const StepDesc* sd, const int64_t* start, int n) {
    const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;   // one warp per trajectory
    if (e >= start[n]) return;
    const int p = find_problem(start, n, e);
    const StepDesc& d = sd[p];
    const int64_t m = e - start[p];
    if (!window_sample(*d.d_t + 1, d.n_window, d.n_stride)) return;
    double sx, sy, sz;
    warp_tile_sums(d.part, d.M, d.n_rt, m, threadIdx.x & 31, sx, sy, sz);
    if ((threadIdx.x & 31) == 0) add_moments(d.mom + 5 * m, sx, sy, sz);
}

__global__ void k_advance_group(const StepDesc* sd, int n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t t1 = *sd[p].d_t + 1;
    if (window_sample(t1, sd[p].n_window, sd[p].n_stride)) *sd[p].d_count += 1;
    *sd[p].d_t = t1;
}

__global__ void k_f32_to_f64_rows(const float* X, const float* Y, const float* Z, double* x, double* y, double* z,
                                  int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    x[e] = X[e];
    y[e] = Y[e];
    z[e] = Z[e];
}

__global__ void k_f64_to_f32_rows(const double* x, const double* y, const double* z, float* X, float* Y, float* Z,
                                  int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    X[e] = (float)x[e];
    Y[e] = (float)y[e];
    Z[e] = (float)z[e];
}

__global__ void k_split_vectors(const double* s, int64_t K, int64_t N, int64_t ldk, __nv_bfloat16* hi,
                                __nv_bfloat16* lo, int tf32) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= K * N) return;
    const int64_t r = e / N, k = e - r * N;
    image_store(hi, lo, r * ldk + k, (float)s[e], true, tf32);
}

__global__ void k_split_vectors_f32(const float* s, int64_t K, int64_t N, int64_t ldk, __nv_bfloat16* hi,
                                    __nv_bfloat16* lo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= K * N) return;
    const int64_t r = e / N, k = e - r * N;
    split_store(hi, lo, r * ldk + k, s[e], true);
}

__global__ void k_widen(const float* a, double* b, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) b[e] = a[e];
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    // resolved once (thread-safe initialisation of a local static)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)p;
        return nullptr;
    }();
    return fn;
}

// 2-D tensor map of an operand image (BF16, or FP32 containers in the TF32
// configuration): inner dimension K (extent kext, row pitch ldk elements), outer
// dimension rows; box (K tile) x box_rows with the K configuration's swizzle.
// Reads outside the extents return zeros.
int make_map(twa_ctx* c, CUtensorMap* map, const void* base, int64_t rows, int64_t kext, int64_t ldk, int box_rows,
             int kc) {
    auto fn = encode_fn();
    if (!fn) return set_error(c, TWA_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)kext, (cuuint64_t)rows};
    const bool f32 = kc == 2;
    cuuint64_t strides[1] = {(cuuint64_t)(ldk * (f32 ? 4 : 2))};
    cuuint32_t box[2] = {(cuuint32_t)kcfg_bk(kc), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE,
                    (kc == 0 || kc == 4) ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(c, TWA_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return TWA_OK;
}

template <int MODE, int NT, int BN, int KC, bool PAIR>
int launch_one(twa_ctx* c, const TcMaps& maps, const TcArgs& a, int64_t n_tiles, const Group& grp) {
    auto kern = k_tc<MODE, NT, BN, KC, PAIR>;
    constexpr int smem = Geo<BN, KC, PAIR>::SMEM;
    static std::atomic<bool> attr{false};   // contexts may be set up from several host threads
    if (!attr.load()) {
        TWA_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr.store(true);
    }
    // the highest launch priority: when the noise draw of a later step runs beside
    // this launch, the block scheduler places this kernel's CTAs first
    static int prio = 1;
    if (prio > 0) {
        int lo = 0, hi = 0;
        TWA_CUDA(c, cudaDeviceGetStreamPriorityRange(&lo, &hi));
        prio = hi;
    }
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cfg.attrs = at;
    if constexpr (!PAIR) {
        const int64_t g = grp.sched ? grp.ctas : (n_tiles < c->tc->num_sms ? n_tiles : c->tc->num_sms);
        cfg.gridDim = dim3((unsigned)g, 1, 1);
        cfg.numAttrs = 1;
    } else {
        // clusters of two CTAs; a schedule's units are clusters
        const int64_t units = grp.sched ? grp.ctas : (n_tiles < c->tc->clusters ? n_tiles : c->tc->clusters);
        at[1].id = cudaLaunchAttributeClusterDimension;
        at[1].val.clusterDim.x = 2;
        at[1].val.clusterDim.y = 1;
        at[1].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(2 * units), 1, 1);
        cfg.numAttrs = 2;
    }
    TWA_CUDA(c, cudaLaunchKernelEx(&cfg, kern, maps, a, grp));
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

// Clusters of two CTAs of the pair kernel that can be resident at once (the
// persistent grid of a pair launch): 0 if the device cannot place one.
template <int NT, int KC>
int pair_clusters_of(twa_ctx* c) {
    auto kern = k_tc<MODE_MIX, NT, 256, KC, true>;
    constexpr int smem = Geo<256, KC, true>::SMEM;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * (c->tc->num_sms / 2)), 1, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int pair_clusters(twa_ctx* c) {
    const TcState* t = c->tc;
    if (t->kc == 3) return t->terms == 2 ? pair_clusters_of<2, 3>(c) : pair_clusters_of<1, 3>(c);
    if (t->kc == 4) return t->terms == 2 ? pair_clusters_of<2, 4>(c) : pair_clusters_of<1, 4>(c);
    if (t->kc == 0)
        return t->terms == 3 ? pair_clusters_of<3, 0>(c) : t->terms == 2 ? pair_clusters_of<2, 0>(c)
                                                                          : pair_clusters_of<1, 0>(c);
    return t->terms == 3 ? pair_clusters_of<3, 1>(c) : t->terms == 2 ? pair_clusters_of<2, 1>(c)
                                                                      : pair_clusters_of<1, 1>(c);
}

// One problem (grp.count = 0) or a group of problems in one persistent launch.
template <int MODE, int NT>
int launch_cfg(twa_ctx* c, const TcMaps& maps, const TcArgs& a, const Group& grp = Group{nullptr, nullptr, 0},
               int64_t group_tiles = 0) {
    const int bn = c->tc->bn, kc = c->tc->kc;
    const bool pair = c->tc->pair != 0;
    const int64_t n_ru = pair ? (a.n_rt + 1) / 2 : a.n_rt;   // row units
    const int64_t n_tiles = grp.count ? group_tiles : n_ru * ((a.n_vec + bn - 1) / bn);
    if (pair) {
        if (bn == 256 && kc == 1) return launch_one<MODE, NT, 256, 1, true>(c, maps, a, n_tiles, grp);
        if (bn == 256 && kc == 3) return launch_one<MODE, NT, 256, 3, true>(c, maps, a, n_tiles, grp);
        if (bn == 256 && kc == 4) return launch_one<MODE, NT, 256, 4, true>(c, maps, a, n_tiles, grp);
        if (bn == 256 && kc == 0) return launch_one<MODE, NT, 256, 0, true>(c, maps, a, n_tiles, grp);
        return set_error(c, TWA_EUNSUPPORTED, "CTA pairs: tile configuration not compiled");
    }
#define TWA_TC_CASE(BN_, KC_) \
    if (bn == BN_ && kc == KC_) return launch_one<MODE, NT, BN_, KC_, false>(c, maps, a, n_tiles, grp);
    TWA_TC_CASE(256, 0)
    TWA_TC_CASE(256, 1)
    TWA_TC_CASE(192, 0)
    TWA_TC_CASE(192, 1)
    TWA_TC_CASE(128, 0)
    TWA_TC_CASE(128, 1)
    TWA_TC_CASE(256, 2)
    TWA_TC_CASE(256, 3)
    TWA_TC_CASE(128, 3)
    TWA_TC_CASE(256, 4)
#undef TWA_TC_CASE
    return set_error(c, TWA_EUNSUPPORTED, "tensor-core tile configuration not compiled");
}

// Standalone L.eta launch with the context's term count (two terms of L against
// the BF16 eta in BF16X3, three in FP32 where eta has a lo image, else one).
int launch_leta(twa_ctx* c, const TcMaps& m, const TcArgs& a) {
    switch (leta_terms(c->tc)) {
        case 3: return launch_cfg<MODE_LETA, 3>(c, m, a);
        case 2: return launch_cfg<MODE_LETA, 2>(c, m, a);
        default: return launch_cfg<MODE_LETA, 1>(c, m, a);
    }
}

TcArgs base_args(twa_ctx* c) {
    TcState* t = c->tc;
    TcArgs a{};
    a.N = t->N;
    a.M = t->M;
    a.ldk = t->ldk;
    a.n_rt = t->n_rt;
    a.n_vec = 2 * t->M;
    a.hdtG = (float)(0.5 * c->dt * c->Gamma);
    a.hdtw = (float)(0.5 * c->dt * t->wsc);
    a.sgdt = (float)sqrt(c->Gamma * c->dt);
    a.sdt = (float)(sqrt(c->dt) * t->lsc);
    a.fsc = 1.0f;
    a.renorm = c->opts.renormalize;
    a.integ = c->opts.integrator;
    a.band = t->band;
    a.flags = c->d_flags;
    return a;
}

int env_int(const char* name, int dflt) {
    const char* v = getenv(name);
    return v ? atoi(v) : dflt;
}

bool pair_capable(const TcState* t) { return t->bn == 256 && t->kc != 2; }

// CTA pairs need a compiled pair configuration and room for at least one
// cluster of two; records how many clusters a persistent pair launch uses.
// Unless TWA_TC_PAIR forces them, a configuration without pairs runs on single
// CTAs instead.
int pair_check(twa_ctx* c) {
    TcState* t = c->tc;
    const bool forced = getenv("TWA_TC_PAIR") != nullptr;
    if (!t->pair) return TWA_OK;
    if (!pair_capable(t)) {
        if (!forced) {
            t->pair = 0;
            return TWA_OK;
        }
        return set_error(c, TWA_EINVAL,
                         "TWA_TC_PAIR runs 256-wide tiles with 32-wide K stages (TWA_TC_KC 1 or 3) in the BF16 precisions");
    }
    const int n = pair_clusters(c);
    if (n < 1) {
        if (!forced) {
            t->pair = 0;
            return TWA_OK;
        }
        return set_error(c, TWA_EUNSUPPORTED, "no cluster of two CTAs of the pair kernel fits on this device");
    }
    t->clusters = n;
    return TWA_OK;
}

// B rows one CTA loads per tile: all BN, or half of them in a CTA pair
int b_box(const TcState* t) { return t->pair ? t->bn / 2 : t->bn; }

int make_state_maps(twa_ctx* c) {
    TcState* t = c->tc;
    int rc;
    const int64_t R = 2 * c->M;
    const int bb = b_box(t);
    // where no lo image is kept (TF32; eta outside the FP32 mode) the lo map
    // aliases the hi image: it is never read (one term)
    if ((rc = make_map(c, &t->tmShi, t->Shi, R, c->N, t->ldk, bb, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmSlo, t->Slo ? t->Slo : t->Shi, R, c->N, t->ldk, bb, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmPhi, t->Phi, R, c->N, t->ldk, bb, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmPlo, t->Plo ? t->Plo : t->Phi, R, c->N, t->ldk, bb, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmE, t->E, R, c->N, t->ldk, bb, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmElo, t->Elo ? t->Elo : t->E, R, c->N, t->ldk, bb, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmE1, t->E1, R, c->N, t->ldk, bb, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmElo1, t->Elo1 ? t->Elo1 : t->E1, R, c->N, t->ldk, bb, t->kc))) return rc;
    return TWA_OK;
}

int make_matrix_maps(twa_ctx* c) {
    TcState* t = c->tc;
    int rc;
    if ((rc = make_map(c, &t->tmWhi, t->Whi, c->N, c->N, t->ldk, BM, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmWlo, t->Wlo ? t->Wlo : t->Whi, c->N, c->N, t->ldk, BM, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmLhi, t->Lhi, c->N, c->N, t->ldk, BM, t->kc))) return rc;
    if ((rc = make_map(c, &t->tmLlo, t->Llo ? t->Llo : t->Lhi, c->N, c->N, t->ldk, BM, t->kc))) return rc;
    return TWA_OK;
}

}  // namespace

int tc_prepare(twa_ctx* c) {
    if (!c->tc) c->tc = new TcState();
    TcState* t = c->tc;
    t->N = c->N;
    t->ldk = (c->N + 7) / 8 * 8;
    t->n_rt = (c->N + BM - 1) / BM;
    // products per entry of W (against the state) and of L (against the noise):
    // BF16X3 and FP32: three for W (hi*hi + hi*lo + lo*hi); L two (BF16X3: the
    // noise is one BF16 value) or three (FP32: the noise is split too). BF16X2:
    // W and L split, their operand one BF16 value: two and two. BF16L2: W one
    // BF16 product, L split: one and two. BF16B: one and one. BF16, TF32: one
    // and one. BF16L2 and BF16B take two products near the diagonal (band).
    switch (c->opts.precision) {
        case TWA_PREC_BF16X3: t->terms = 3; t->lterms = 2; break;
        case TWA_PREC_FP32: t->terms = 3; t->lterms = 3; break;
        case TWA_PREC_BF16X2: t->terms = 2; t->lterms = 2; break;
        case TWA_PREC_BF16L2: t->terms = 1; t->lterms = 2; break;
        case TWA_PREC_BF16B: t->terms = 1; t->lterms = 1; break;
        default: t->terms = 1; t->lterms = 1; break;
    }
    // BF16L2 (W) and BF16B (W and L): hi + lo within 64 columns of the diagonal
    // (TWA_TC_BAND blocks of 64 on each side of each 256-row unit; 0 = one
    // product everywhere), hi alone beyond: the largest entries, whose rounding
    // errors would add up to the same one-signed error on every row of the
    // Toeplitz W (and of its Cholesky factor, whose rows converge to one
    // sequence), keep ~16 bits, at ~3 % more products than one per entry
    const bool banded = c->opts.precision == TWA_PREC_BF16L2 || c->opts.precision == TWA_PREC_BF16B;
    t->band = banded ? env_int("TWA_TC_BAND", 1) : 0;
    if (t->band < 0 || t->band > 64) return set_error(c, TWA_EINVAL, "TWA_TC_BAND must be in 0 .. 64");
    // tile configuration: TWA_TC_BN in {128, 192, 256}, TWA_TC_KC in {0, 1, 3, 4}
    // (3: at most two products per entry, BN 128 or 256; 4: the same with 64-wide
    // K stages and 128-byte swizzle, BN 256).
    // Defaults measured fastest at N = 10^4, M = 1024 (same-box A/B, all bit-identical):
    // 256-wide tiles on CTA pairs with 64-wide K stages and 128-byte swizzle -- one
    // operand image per stage for the precisions with at most two products (KC = 4;
    // BF16X2: 1.63 ms/step against 1.83 for single CTAs with six 32-wide stages),
    // four images otherwise (KC = 0; BF16X3: 2.15 against 2.45 ms). On single CTAs
    // the 32-wide four-image stage is faster for BF16X3 (KC = 1). The TF32 and FP32
    // precisions have one configuration: 256-wide tiles, four 16-wide FP32 K stages
    // (KC = 2).
    const bool tf32 = c->opts.precision == TWA_PREC_TF32 || c->opts.precision == TWA_PREC_FP32;
    if (tf32 && (getenv("TWA_TC_BN") || getenv("TWA_TC_KC")))
        return set_error(c, TWA_EINVAL, "TWA_TC_BN / TWA_TC_KC do not apply to the TF32 and FP32 precisions");
    t->bn = tf32 ? 256 : env_int("TWA_TC_BN", 256);
    const bool one_b = t->terms <= 2 && t->lterms <= 2;
    const int kc_default = one_b ? (t->bn == 256 ? 4 : t->bn == 128 ? 3 : 1) : (t->bn == 256 ? 0 : 1);
    t->kc = tf32 ? 2 : env_int("TWA_TC_KC", kc_default);
    // TWA_SEPARATE_LETA=1: dense step as separate noise, L.eta, predictor and
    // corrector launches instead of the two mixed launches (same results)
    t->separate_leta = env_int("TWA_SEPARATE_LETA", 0) != 0;
    t->overlap_noise = env_int("TWA_NOISE_OVERLAP", 1) != 0;
    // TWA_NOISE_EPILOGUE=0: the dense step's noise draw as its own kernel (on a
    // second stream unless TWA_NOISE_OVERLAP=0) instead of inside the MIX launches
    t->noise_epi = env_int("TWA_NOISE_EPILOGUE", 1) != 0;
    if (!tf32 &&
        (!(t->bn == 128 || t->bn == 192 || t->bn == 256) || !(t->kc == 0 || t->kc == 1 || t->kc == 3 || t->kc == 4)))
        return set_error(c, TWA_EINVAL, "TWA_TC_BN must be 128, 192 or 256 and TWA_TC_KC 0, 1, 3 or 4");
    if (t->kc == 3 && (t->terms > 2 || t->lterms > 2 || t->bn == 192))
        return set_error(c, TWA_EINVAL, "TWA_TC_KC = 3 holds one operand image: at most two products, BN 128 or 256");
    if (t->kc == 4 && (t->terms > 2 || t->lterms > 2 || t->bn != 256))
        return set_error(c, TWA_EINVAL, "TWA_TC_KC = 4 holds one operand image: at most two products, BN 256");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess && sms > 0)
        t->num_sms = sms;
    // CTA pairs (256-row tiles on clusters of two, tcgen05 cta_group::2) wherever a
    // pair configuration is compiled: the BF16 precisions with 256-wide tiles and
    // 32-wide K stages (same-box A/B at N = 10^4, BF16X2: 3 % faster per step, same
    // bits). TWA_TC_PAIR=0 / 1 forces them off / on.
    t->pair = env_int("TWA_TC_PAIR", pair_capable(t) ? 1 : 0) != 0;
    if (int rc = pair_check(c)) return rc;
    if (!t->pair && !getenv("TWA_TC_KC") && t->kc == 0) t->kc = 1;   // the single-CTA default
    const size_t nb = (size_t)(tf32 ? 4 : 2) * c->N * t->ldk;
    __nv_bfloat16** m4[] = {&t->Whi, &t->Lhi, &t->Wlo, &t->Llo};
    for (int k = 0; k < (tf32 && t->terms == 1 ? 2 : 4); ++k)
        if (dev_malloc(c, m4[k], nb) != cudaSuccess) return set_error(c, TWA_ENOMEM, "device operand images");
    const unsigned g = nblk(c->N * t->ldk, 256) > 8192 ? 8192 : nblk(c->N * t->ldk, 256);
    // W = w W1 and L = sqrt(w) L1 with W1, L1 independent of w: the images hold W1
    // and L1 and the epilogues apply w and sqrt(w), so runs at w (1 +- delta) differ
    // only in those two FP32 factors (finite differences in w see no image rounding)
    t->wsc = c->w > 0.0 ? c->w : 1.0;
    t->lsc = c->w > 0.0 ? sqrt(c->w) : 1.0;
    k_split_matrix<<<g, 256, 0, c->stream>>>(c->W64, c->N, t->ldk, t->Whi, t->Wlo, tf32, 1.0 / t->wsc);
    k_split_matrix<<<g, 256, 0, c->stream>>>(c->L64, c->N, t->ldk, t->Lhi, t->Llo, tf32, 1.0 / t->lsc);
    TWA_CUDA(c, cudaGetLastError());
    return make_matrix_maps(c);
}

int tc_alloc(twa_ctx* c) {
    TcState* t = c->tc;
    t->M = c->M;
    const size_t mn = (size_t)c->M * c->N;
    float** f[] = {&t->X, &t->Y, &t->Z, &t->Xp, &t->Yp, &t->Zp, &t->Bx, &t->By};
    for (auto p : f)
        if (dev_malloc(c, p, sizeof(float) * mn) != cudaSuccess) return set_error(c, TWA_ENOMEM, "device state");
    // FP32 containers in the TF32 and FP32 modes; lo images of s and s~ except in
    // TF32, and of eta in FP32 only
    const bool tf32 = t->kc == 2;
    const size_t ni = (size_t)(tf32 ? 4 : 2) * 2 * (size_t)c->M * t->ldk;
    __nv_bfloat16** b[] = {&t->Shi, &t->Phi, &t->E, &t->Slo, &t->Plo, &t->Elo};
    const int nimg = !tf32 ? 5 : t->terms == 3 ? 6 : 3;
    for (int k = 0; k < nimg; ++k) {
        if (dev_malloc(c, b[k], ni) != cudaSuccess) return set_error(c, TWA_ENOMEM, "device images");
        TWA_CUDA(c, cudaMemsetAsync(*b[k], 0, ni, c->stream));
    }
    // the odd-step noise buffers (dense route; the FFT route draws into E only)
    if (dev_malloc(c, &t->E1, ni) != cudaSuccess) return set_error(c, TWA_ENOMEM, "device images");
    TWA_CUDA(c, cudaMemsetAsync(t->E1, 0, ni, c->stream));
    if (t->Elo) {
        if (dev_malloc(c, &t->Elo1, ni) != cudaSuccess) return set_error(c, TWA_ENOMEM, "device images");
        TWA_CUDA(c, cudaMemsetAsync(t->Elo1, 0, ni, c->stream));
    }
    if (dev_malloc(c, &t->XI, sizeof(float) * 2 * c->M) != cudaSuccess ||
        dev_malloc(c, &t->XI1, sizeof(float) * 2 * c->M) != cudaSuccess ||
        dev_malloc(c, &t->part, sizeof(float) * 4 * c->M * t->n_rt) != cudaSuccess ||
        dev_malloc(c, &t->partp, sizeof(float) * 4 * c->M * t->n_rt) != cudaSuccess)
        return set_error(c, TWA_ENOMEM, "device sums");
    return make_state_maps(c);
}

namespace {
void mix_free(TcState* t);
}

void tc_free_run(twa_ctx* c) {
    TcState* t = c->tc;
    if (!t) return;
    mix_free(t);
    float** f[] = {&t->X, &t->Y, &t->Z, &t->Xp, &t->Yp, &t->Zp, &t->Bx, &t->By, &t->Bx1,
                   &t->By1, &t->XI, &t->XI1, &t->part, &t->partp};
    for (auto p : f) {
        dev_free(c, *p);
        *p = nullptr;
    }
    __nv_bfloat16** b[] = {&t->Shi, &t->Slo, &t->Phi, &t->Plo, &t->E, &t->Elo, &t->E1, &t->Elo1};
    for (auto p : b) {
        dev_free(c, *p);
        *p = nullptr;
    }
}

int tc_set_extra_matrix(twa_ctx* c, int slot, const double* A64) {
    TcState* t = c->tc;
    if (slot < 0 || slot > 1) return set_error(c, TWA_EINVAL, "tc_set_extra_matrix: slot");
    if (t->kc == 2) return set_error(c, TWA_EUNSUPPORTED, "extra matrices run on the BF16 precisions");
    const size_t nb = sizeof(__nv_bfloat16) * (size_t)c->N * t->ldk;
    if (!t->Xhi[slot]) {
        if (dev_malloc(c, &t->Xhi[slot], nb) != cudaSuccess || dev_malloc(c, &t->Xlo[slot], nb) != cudaSuccess)
            return set_error(c, TWA_ENOMEM, "device extra matrix images");
    }
    const unsigned g = nblk(c->N * t->ldk, 256) > 8192 ? 8192 : nblk(c->N * t->ldk, 256);
    k_split_matrix<<<g, 256, 0, c->stream>>>(A64, c->N, t->ldk, t->Xhi[slot], t->Xlo[slot], 0, 1.0);
    TWA_CUDA(c, cudaGetLastError());
    int rc;
    if ((rc = make_map(c, &t->tmXhi[slot], t->Xhi[slot], c->N, c->N, t->ldk, BM, t->kc))) return rc;
    return make_map(c, &t->tmXlo[slot], t->Xlo[slot], c->N, c->N, t->ldk, BM, t->kc);
}

int tc_contract_f32(twa_ctx* c, int which, const float* in, float* out, int64_t K) {
    TcState* t = c->tc;
    int rc;
    if (t->kc == 2) return set_error(c, TWA_EUNSUPPORTED, "FP32 contractions run on the BF16 precisions");
    if (t->vec_rows != K) {
        dev_free(c, t->Vhi);
        dev_free(c, t->Vlo);
        const size_t ni = sizeof(__nv_bfloat16) * (size_t)K * t->ldk;
        t->Vhi = t->Vlo = nullptr;
        if (dev_malloc(c, &t->Vhi, ni) != cudaSuccess || dev_malloc(c, &t->Vlo, ni) != cudaSuccess)
            return set_error(c, TWA_ENOMEM, "device vector images");
        TWA_CUDA(c, cudaMemsetAsync(t->Vhi, 0, ni, c->stream));
        TWA_CUDA(c, cudaMemsetAsync(t->Vlo, 0, ni, c->stream));
        if ((rc = make_map(c, &t->tmVhi, t->Vhi, K, c->N, t->ldk, b_box(t), t->kc))) return rc;
        if ((rc = make_map(c, &t->tmVlo, t->Vlo, K, c->N, t->ldk, b_box(t), t->kc))) return rc;
        t->vec_rows = K;
    }
    k_split_vectors_f32<<<nblk(K * c->N, 256), 256, 0, c->stream>>>(in, K, c->N, t->ldk, t->Vhi, t->Vlo);
    TcMaps m{};
    if (which == 0) { m.a0 = t->tmWhi; m.a1 = t->tmWlo; }
    else if (which == 1) { m.a0 = t->tmLhi; m.a1 = t->tmLlo; }
    else if ((which == 2 || which == 3) && t->Xhi[which - 2]) { m.a0 = t->tmXhi[which - 2]; m.a1 = t->tmXlo[which - 2]; }
    else return set_error(c, TWA_EINVAL, "tc_contract_f32: unknown operand");
    m.b0 = t->tmVhi;
    m.b1 = t->tmVlo;
    TcArgs a = base_args(c);
    a.n_vec = K;
    a.field_out = out;
    a.fsc = which == 0 ? (float)t->wsc : which == 1 ? (float)t->lsc : 1.0f;   // extra matrices: unscaled images
    // L and dL/dalpha against the noise: the step's L.eta product count
    const int nterms = (which == 1 || which == 3) ? leta_terms(t) : t->terms;
    return nterms == 3   ? launch_cfg<MODE_FIELD, 3>(c, m, a)
           : nterms == 2 ? launch_cfg<MODE_FIELD, 2>(c, m, a)
                         : launch_cfg<MODE_FIELD, 1>(c, m, a);
}

void tc_free(twa_ctx* c) {
    TcState* t = c->tc;
    if (!t) return;
    tc_free_run(c);
    if (t->side) {
        cudaStreamSynchronize(t->side);
        cudaStreamDestroy(t->side);
    }
    if (t->ev_fork) cudaEventDestroy(t->ev_fork);
    if (t->ev_join) cudaEventDestroy(t->ev_join);
    void* extra[] = {t->Xhi[0], t->Xhi[1], t->Xlo[0], t->Xlo[1], t->Vhi, t->Vlo};
    for (void* p : extra) dev_free(c, p);
    void* all[] = {t->Whi, t->Wlo, t->Lhi, t->Llo};
    for (void* p : all) dev_free(c, p);
    delete t;
    c->tc = nullptr;
}

int tc_state_changed(twa_ctx* c) {
    TcState* t = c->tc;
    t->bn_ready = -1;
    const int64_t MN = c->M * c->N;
    k_images_tc<<<nblk(MN, 256), 256, 0, c->stream>>>(t->X, t->Y, t->Shi, t->Slo, c->M, c->N, t->ldk, t->kc == 2);
    k_part_tc<<<nblk(t->n_rt * c->M, 8), 256, 0, c->stream>>>(t->X, t->Y, t->Z, t->part, c->M, c->N, t->n_rt);
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

int tc_init_state(twa_ctx* c) {
    TcState* t = c->tc;
    t->bn_ready = -1;
    k_init_tc<<<nblk(c->M * c->N, 256), 256, 0, c->stream>>>(t->X, t->Y, t->Z, t->Shi, t->Slo, c->M, c->N, t->ldk,
                                                            c->seed, (float)c->opts.init_state,
                                                            c->opts.traj_offset, t->kc == 2);
    TWA_CUDA(c, cudaGetLastError());
    k_part_tc<<<nblk(t->n_rt * c->M, 8), 256, 0, c->stream>>>(t->X, t->Y, t->Z, t->part, c->M, c->N, t->n_rt);
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

// ---------------------------------------------------------------------------
// the dense step as two mixed persistent launches

// Descriptor tables and tile schedules of the dense step. Launch 0 holds the
// predictor of step t, launch 1 its corrector; each also takes a share of the
// L.eta tiles of step t + 1 (the noise part depends only on that step's noise),
// so the triangular L.eta needs no launch of its own and fills the tails of the
// two W.s launches.
struct MixPlan {
    int nprob = 0;                            // 3 x problems: predictor, corrector, L.eta blocks
    GroupDesc* desc = nullptr;                // [parity of t][predictor | corrector | L.eta][problem]
    int64_t* start = nullptr;                 // [nprob + 1] first flat tile of each problem
    int64_t* lstart = nullptr;                // [problems + 1] tile prefix within the L.eta block
    int32_t* list[2] = {nullptr, nullptr};    // per launch: flat tiles, CTA after CTA
    int32_t* first[2] = {nullptr, nullptr};   // per launch: [ctas + 1] offsets into list
    int ctas[2] = {0, 0};
    int64_t tiles[2] = {0, 0};
    double flops[2] = {0.0, 0.0};             // tensor-core FLOPs issued per launch
    double alg[2] = {0.0, 0.0};               // algorithmic FLOPs per launch (counted once)
    double leta_flops = 0.0, w_flops = 0.0;   // issued: all L.eta tiles / all W.s tiles of one stage
    double leta_alg = 0.0, w_alg = 0.0;       // algorithmic: the same
    int64_t leta_tiles = 0;                   // tiles of the L.eta block
    std::vector<GroupDesc> host;              // host copy of desc
    twa_ctx* owner = nullptr;                 // whose allocator the tables came from
};

namespace {

void mix_plan_free(MixPlan* p) {
    if (!p) return;
    void* q[] = {p->desc, p->start, p->lstart, p->list[0], p->list[1], p->first[0], p->first[1]};
    for (void* x : q) dev_free(p->owner, x);
    delete p;
}

void mix_free(TcState* t) {
    mix_plan_free(t->mix);
    t->mix = nullptr;
    t->bn_ready = -1;
}

// Longest-processing-time list scheduling: the tiles, longest first, each to
// the CTA with the least work so far (ties to the lower CTA index); a CTA runs
// its tiles in the order received. Returns the largest CTA load.
int64_t lpt_schedule(std::vector<std::pair<int64_t, int32_t>> jobs, int ctas, std::vector<int32_t>* list,
                     std::vector<int32_t>* first) {
    std::stable_sort(jobs.begin(), jobs.end(),
                     [](const std::pair<int64_t, int32_t>& a, const std::pair<int64_t, int32_t>& b) {
                         return a.first > b.first;
                     });
    using Load = std::pair<int64_t, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < ctas; ++b) heap.push({0, b});
    std::vector<std::vector<int32_t>> per(list ? ctas : 0);
    for (const auto& j : jobs) {
        Load l = heap.top();
        heap.pop();
        if (list) per[l.second].push_back(j.second);
        heap.push({l.first + j.first, l.second});
    }
    int64_t span = 0;
    while (!heap.empty()) {
        span = std::max(span, heap.top().first);
        heap.pop();
    }
    if (list) {
        list->clear();
        first->assign(1, 0);
        for (int b = 0; b < ctas; ++b) {
            list->insert(list->end(), per[b].begin(), per[b].end());
            first->push_back((int32_t)list->size());
        }
    }
    return span;
}

// Descriptor table and the two launches' tile schedules of the dense step for
// n problems advanced together (n = 1: one context; n > 1: a batched scan). Per
// parity of the step index, the table holds the W.s + predictor problems, the
// W.s~ + corrector problems and the L.eta problems of step t + 1; launch 1 runs
// the predictor tiles and the longest L.eta tiles, launch 2 the corrector tiles
// and the rest, each placed on the CTAs by longest-first list scheduling.
int mix_plan_build(twa_ctx* const* cs, int n, twa_ctx* ec, MixPlan* p) {
    const TcState* t0 = cs[0]->tc;
    const int bn = t0->bn, bk = kcfg_bk(t0->kc);
    const int ntw = t0->terms, ntl = leta_terms(t0);
    // tiles are (row unit, column tile) pairs; a row unit is one 128-row tile, or
    // two on a CTA pair, and the scheduling units are CTAs or clusters of two
    const bool pair = t0->pair != 0;
    const int64_t bmu = pair ? 2 * BM : BM;
    auto units_of = [&](int64_t n_rt) { return pair ? (n_rt + 1) / 2 : n_rt; };
    const int nprob = 3 * n;
    p->nprob = nprob;
    // flat tile ranges: [W.s + predictor of 0..n-1][W.s~ + corrector][L.eta]
    std::vector<int64_t> st(nprob + 1, 0), nct(n), nk(n);
    for (int q = 0; q < n; ++q) {
        const TcState* t = cs[q]->tc;
        nct[q] = (2 * cs[q]->M + bn - 1) / bn;
        nk[q] = (cs[q]->N + bk - 1) / bk;
        const int64_t T = units_of(t->n_rt) * nct[q];
        st[q + 1] = T;
        st[n + q + 1] = T;
        st[2 * n + q + 1] = T;
    }
    for (int k = 0; k < nprob; ++k) st[k + 1] += st[k];
    if (st[nprob] > INT32_MAX) return set_error(ec, TWA_EUNSUPPORTED, "dense step: too many tiles");
    for (int q = 0; q < n; ++q) {
        TcState* t = cs[q]->tc;
        const size_t mn = sizeof(float) * cs[q]->M * cs[q]->N;
        if (!t->Bx1 && (dev_malloc(cs[q], &t->Bx1, mn) != cudaSuccess || dev_malloc(cs[q], &t->By1, mn) != cudaSuccess))
            return set_error(ec, TWA_ENOMEM, "device noise part");
    }

    // tile costs in K stages x products; FLOPs issued and algorithmic per tile
    std::vector<std::pair<int64_t, int32_t>> pjobs, cjobs, ljobs;
    std::vector<double> fl(st[nprob]), fa(st[nprob]);
    for (int q = 0; q < n; ++q) {
        const int64_t N = cs[q]->N, M = cs[q]->M, n_ru = units_of(cs[q]->tc->n_rt);
        auto rows_of = [&](int64_t ru) { return std::min<int64_t>(bmu, N - ru * bmu); };
        auto cols_of = [&](int64_t ct) { return (double)std::min<int64_t>(bn, 2 * M - ct * bn); };
        const int band = cs[q]->tc->band;
        for (int64_t x = 0; x < st[q + 1] - st[q]; ++x) {
            const int64_t rt = x / nct[q], ct = x - rt * nct[q];
            // one-product W: its two-product band adds stages and K columns
            int64_t kx = 0, cx = 0;
            if (ntw == 1 && band > 0) {
                int kb0, kb1;
                two_product_stages(rt, (int)bmu, bk, band, kb0, kb1);
                const int64_t a = std::max<int64_t>(kb0, 0), b = std::min<int64_t>(kb1, nk[q]);
                if (b > a) {
                    kx = b - a;
                    cx = std::min<int64_t>(b * bk, N) - a * bk;
                }
            }
            const double f = 2.0 * rows_of(rt) * (double)(N * ntw + cx) * cols_of(ct);
            pjobs.push_back({nk[q] * ntw + kx, (int32_t)(st[q] + x)});
            cjobs.push_back({nk[q] * ntw + kx, (int32_t)(st[n + q] + x)});
            fl[st[q] + x] = fl[st[n + q] + x] = f;
            fa[st[q] + x] = fa[st[n + q] + x] = 2.0 * rows_of(rt) * (double)N * cols_of(ct);
            // the kernel hands out L.eta row units longest first
            const int64_t lrt = n_ru - 1 - rt;
            const int64_t k1 = std::min<int64_t>((lrt * bmu + bmu + bk - 1) / bk, nk[q]);
            const double r0 = (double)(lrt * bmu), r1 = r0 + rows_of(lrt);
            int64_t lkx = 0, lcx = 0;
            if (ntl == 1 && band > 0) {
                int kb0, kb1;
                two_product_stages(lrt, (int)bmu, bk, band, kb0, kb1);
                const int64_t a = std::max<int64_t>(kb0, 0), b = std::min<int64_t>(kb1, k1);
                if (b > a) {
                    lkx = b - a;
                    lcx = std::min<int64_t>(b * bk, N) - a * bk;
                }
            }
            ljobs.push_back({k1 * ntl + lkx, (int32_t)(st[2 * n + q] + x)});
            fa[st[2 * n + q] + x] = 2.0 * ((r1 * (r1 + 1) - r0 * (r0 + 1)) / 2.0) * cols_of(ct);   // triangle
            fl[st[2 * n + q] + x] = fa[st[2 * n + q] + x] * ntl + 2.0 * rows_of(lrt) * (double)lcx * cols_of(ct);
        }
    }
    std::stable_sort(ljobs.begin(), ljobs.end(),
                     [](const std::pair<int64_t, int32_t>& a, const std::pair<int64_t, int32_t>& b) {
                         return a.first > b.first;
                     });
    // the predictor's launch takes the kl longest L.eta tiles, the corrector's the rest
    const int sms = pair ? t0->clusters : t0->num_sms;
    auto ctas_for = [&](int64_t k) { return (int)std::min<int64_t>(k, sms); };
    const int64_t Tl = (int64_t)ljobs.size();
    auto span_of = [&](int64_t kl) {
        std::vector<std::pair<int64_t, int32_t>> a(pjobs), b(cjobs);
        a.insert(a.end(), ljobs.begin(), ljobs.begin() + kl);
        b.insert(b.end(), ljobs.begin() + kl, ljobs.end());
        return lpt_schedule(a, ctas_for((int64_t)a.size()), nullptr, nullptr) +
               lpt_schedule(b, ctas_for((int64_t)b.size()), nullptr, nullptr);
    };
    // coarse search over 32 split points, then a finer one around the best
    int64_t best_k = 0, best = span_of(0);
    auto scan = [&](int64_t lo, int64_t hi, int64_t stride) {
        for (int64_t kl = lo; kl <= hi; kl += stride) {
            const int64_t s = span_of(kl);
            if (s < best) best = s, best_k = kl;
        }
    };
    const int64_t coarse = std::max<int64_t>(1, Tl / 32);
    scan(coarse, Tl, coarse);
    const int64_t fine = std::max<int64_t>(1, coarse / 16);
    scan(std::max<int64_t>(0, best_k - coarse), std::min<int64_t>(Tl, best_k + coarse), fine);

    std::vector<int32_t> lists[2], firsts[2];
    std::vector<int> seen(st[nprob], 0);
    for (int L = 0; L < 2; ++L) {
        std::vector<std::pair<int64_t, int32_t>> jobs(L == 0 ? pjobs : cjobs);
        if (L == 0) jobs.insert(jobs.end(), ljobs.begin(), ljobs.begin() + best_k);
        else jobs.insert(jobs.end(), ljobs.begin() + best_k, ljobs.end());
        p->ctas[L] = ctas_for((int64_t)jobs.size());
        p->tiles[L] = (int64_t)jobs.size();
        lpt_schedule(jobs, p->ctas[L], &lists[L], &firsts[L]);
        // each CTA walks its tiles in flat order: a problem's tiles stay together
        // (fewer descriptor switches, W rows reused while in L2)
        for (int c = 0; c < p->ctas[L]; ++c)
            std::sort(lists[L].begin() + firsts[L][c], lists[L].begin() + firsts[L][c + 1]);
        for (int32_t x : lists[L]) {
            p->flops[L] += fl[x];
            p->alg[L] += fa[x];
            ++seen[x];
        }
    }
    for (int64_t x = st[2 * n]; x < st[nprob]; ++x) {
        p->leta_flops += fl[x];
        p->leta_alg += fa[x];
    }
    p->leta_tiles = st[nprob] - st[2 * n];
    for (int64_t x = 0; x < st[n]; ++x) {
        p->w_flops += fl[x];
        p->w_alg += fa[x];
    }
    // every tile in exactly one launch
    for (int64_t x = 0; x < st[nprob]; ++x)
        if (seen[x] != 1) return set_error(ec, TWA_EUNSUPPORTED, "dense step: internal error in the tile schedule");

    // descriptors: [parity of t][predictor | corrector | L.eta][problem]
    std::vector<GroupDesc> d(2 * nprob);
    for (int par = 0; par < 2; ++par) {
        for (int q = 0; q < n; ++q) {
            twa_ctx* c = cs[q];
            TcState* t = c->tc;
            float* bx = par ? t->Bx1 : t->Bx;   // noise part of step t (this parity)
            float* by = par ? t->By1 : t->By;
            float* nx = par ? t->Bx : t->Bx1;   // ... and of step t + 1
            float* ny = par ? t->By : t->By1;
            TcArgs la = base_args(c), pa = base_args(c), ca = base_args(c);
            la.flags = pa.flags = ca.flags = ec->d_flags;
            la.XI = par ? t->XI : t->XI1;       // collective normals of step t + 1
            la.oBnx = nx;
            la.oBny = ny;
            pa.X = t->X; pa.Y = t->Y; pa.Z = t->Z;
            pa.Bnx = bx; pa.Bny = by;
            pa.oX = t->Xp; pa.oY = t->Yp; pa.oZ = t->Zp;
            pa.oHi = t->Phi; pa.oLo = t->Plo;
            pa.part_in = t->part; pa.part_out = t->partp;
            // the midpoint scheme's corrector rotates s itself (in place)
            const bool mid = c->opts.integrator == TWA_INT_MIDPOINT;
            ca.X = mid ? t->X : t->Xp; ca.Y = mid ? t->Y : t->Yp; ca.Z = mid ? t->Z : t->Zp;
            ca.X0 = t->X; ca.Y0 = t->Y; ca.Z0 = t->Z;
            ca.Bnx = bx; ca.Bny = by;
            ca.oX = t->X; ca.oY = t->Y; ca.oZ = t->Z;
            ca.oHi = t->Shi; ca.oLo = t->Slo;
            ca.part_in = t->partp; ca.part_out = t->part;
            GroupDesc* g = &d[par * nprob];
            g[q] = GroupDesc{TcMaps{t->tmWhi, t->tmWlo, t->tmShi, t->tmSlo}, pa, MODE_PRED, ntw};
            g[n + q] = GroupDesc{TcMaps{t->tmWhi, t->tmWlo, t->tmPhi, t->tmPlo}, ca, MODE_CORR, ntw};
            // L.eta of step t + 1: its noise images are E (t + 1 even) or E1 (odd)
            g[2 * n + q] = GroupDesc{TcMaps{t->tmLhi, t->tmLlo, par ? t->tmE : t->tmE1, par ? t->tmElo : t->tmElo1},
                                     la, MODE_LETA, ntl};
        }
    }
    p->host = d;
    std::vector<int64_t> lst(n + 1);
    for (int q = 0; q <= n; ++q) lst[q] = st[2 * n + q] - st[2 * n];
    p->owner = ec;
    bool ok = dev_malloc(ec, &p->desc, sizeof(GroupDesc) * d.size()) == cudaSuccess &&
              dev_malloc(ec, &p->start, sizeof(int64_t) * st.size()) == cudaSuccess &&
              dev_malloc(ec, &p->lstart, sizeof(int64_t) * lst.size()) == cudaSuccess;
    for (int L = 0; L < 2 && ok; ++L)
        ok = dev_malloc(ec, &p->list[L], sizeof(int32_t) * lists[L].size()) == cudaSuccess &&
             dev_malloc(ec, &p->first[L], sizeof(int32_t) * firsts[L].size()) == cudaSuccess;
    if (!ok) return set_error(ec, TWA_ENOMEM, "device allocation of the dense step plan");
    ok = cudaMemcpy(p->desc, d.data(), sizeof(GroupDesc) * d.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(p->start, st.data(), sizeof(int64_t) * st.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(p->lstart, lst.data(), sizeof(int64_t) * lst.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    for (int L = 0; L < 2 && ok; ++L)
        ok = cudaMemcpy(p->list[L], lists[L].data(), sizeof(int32_t) * lists[L].size(), cudaMemcpyHostToDevice) ==
                 cudaSuccess &&
             cudaMemcpy(p->first[L], firsts[L].data(), sizeof(int32_t) * firsts[L].size(),
                        cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) return set_error(ec, TWA_ECUDA, "dense step plan upload failed");
    return TWA_OK;
}

int mix_build(twa_ctx* c) {
    MixPlan* p = new MixPlan();
    c->tc->mix = p;
    twa_ctx* cs[1] = {c};
    return mix_plan_build(cs, 1, c, p);
}

}  // namespace

static bool tc_mixed_step(const twa_ctx* c) { return c->tc && !c->fft; }

namespace {
// The second stream (lowest priority) and the fork / join events of the noise draw.
int side_stream(twa_ctx* c) {
    TcState* ts = c->tc;
    if (ts->side) return TWA_OK;
    int lo = 0, hi = 0;
    TWA_CUDA(c, cudaDeviceGetStreamPriorityRange(&lo, &hi));
    TWA_CUDA(c, cudaStreamCreateWithPriority(&ts->side, cudaStreamNonBlocking, lo));
    TWA_CUDA(c, cudaEventCreateWithFlags(&ts->ev_fork, cudaEventDisableTiming));
    TWA_CUDA(c, cudaEventCreateWithFlags(&ts->ev_join, cudaEventDisableTiming));
    return TWA_OK;
}

// Noise of step t (= *d_t) and its noise part, by a standalone L.eta launch,
// into the buffer of the step's parity.
int noise_part_alone(twa_ctx* c, int64_t t) {
    TcState* ts = c->tc;
    {
        ProfScope p(c, TWA_PROF_NOISE);
        k_noise_tc<<<nblk(c->M * (c->N + 1), 256), 256, 0, c->stream>>>(
            ts->E, ts->Elo, ts->XI, ts->E1, ts->Elo1, ts->XI1, c->M, c->N, ts->ldk, c->seed, c->d_t, 0,
            c->opts.traj_offset, ts->kc == 2);
    }
    const bool odd = t & 1;
    TcArgs la = base_args(c);
    la.XI = odd ? ts->XI1 : ts->XI;
    la.oBnx = odd ? ts->Bx1 : ts->Bx;
    la.oBny = odd ? ts->By1 : ts->By;
    const TcMaps lm{ts->tmLhi, ts->tmLlo, odd ? ts->tmE1 : ts->tmE, odd ? ts->tmElo1 : ts->tmElo};
    ProfScope p(c, TWA_PROF_NOISE_FACTOR, ts->mix->leta_flops, ts->mix->leta_alg);
    return launch_leta(c, lm, la);
}
}  // namespace

// Noise part of step t into its buffer and the noise of step t + 1 into its
// images, unless already there (after step t - 1 both are).
int tc_prime(twa_ctx* c, int64_t t) {
    TcState* ts = c->tc;
    if (!tc_mixed_step(c) || ts->separate_leta || ts->bn_ready == t) return TWA_OK;
    int rc;
    if (!ts->mix && (rc = mix_build(c))) return rc;
    if ((rc = noise_part_alone(c, t))) return rc;
    // and the noise of step t + 1, which step t's L.eta tiles read
    k_noise_tc<<<nblk(c->M * (c->N + 1), 256), 256, 0, c->stream>>>(ts->E, ts->Elo, ts->XI, ts->E1, ts->Elo1, ts->XI1,
                                                                    c->M, c->N, ts->ldk, c->seed, c->d_t, 1,
                                                                    c->opts.traj_offset, ts->kc == 2);
    TWA_CUDA(c, cudaGetLastError());
    ts->bn_ready = t;
    return TWA_OK;
}

void tc_steps_done(twa_ctx* c, int64_t t_next) {
    if (tc_mixed_step(c)) c->tc->bn_ready = t_next;
}

// Launches of step t alone, with no host-side bookkeeping (so that they can be
// captured into a graph). The dense route needs the noise part of step t in its
// buffer (tc_prime) and leaves that of step t + 1 in the other.
int tc_launch_step(twa_ctx* c, int64_t t) {
    TcState* ts = c->tc;
    const int64_t M = c->M, N = c->N;
    const int ntw = ts->terms;
    int rc;
    if (c->fft) {
        // Toeplitz route: W.s by FFT with the Heun update in the same kernel; the
        // noise part from L.eta, or from one transform of the circulant embedding
        if (c->opts.noise_route == TWA_NOISE_CIRCULANT) {
            ProfScope p(c, TWA_PROF_NOISE);
            rc = fft_noise(c);
        } else {
            {
                ProfScope p(c, TWA_PROF_NOISE);
                k_noise_tc<<<nblk(M * (N + 1), 256), 256, 0, c->stream>>>(ts->E, ts->Elo, ts->XI, ts->E, ts->Elo,
                                                                         ts->XI, M, N, ts->ldk, c->seed, c->d_t, 0,
                                                                         c->opts.traj_offset, ts->kc == 2);
            }
            TcArgs la = base_args(c);
            la.XI = ts->XI;
            la.oBnx = ts->Bx;
            la.oBny = ts->By;
            const TcMaps lm{ts->tmLhi, ts->tmLlo, ts->tmE, ts->tmElo};
            ProfScope p(c, TWA_PROF_NOISE_FACTOR);
            rc = launch_leta(c, lm, la);
        }
        if (rc) return rc;
        {
            ProfScope p(c, TWA_PROF_PREDICT);
            rc = fft_predict(c);
        }
        if (rc) return rc;
        {
            ProfScope p(c, TWA_PROF_CORRECT);
            rc = fft_correct(c);
        }
        return rc;
    }
    if (!ts->mix && (rc = mix_build(c))) return rc;
    MixPlan* mp = ts->mix;
    if (ts->separate_leta) {
        // the same tiles as four separate launches: noise, L.eta, W.s + predictor,
        // W.s~ + corrector (bit-identical results)
        if ((rc = noise_part_alone(c, t))) return rc;
        const GroupDesc* h = mp->host.data() + 3 * (t & 1);   // predictor, corrector, L.eta
        {
            ProfScope p(c, TWA_PROF_PREDICT, mp->w_flops, mp->w_alg);
            rc = ntw == 3   ? launch_cfg<MODE_PRED, 3>(c, h[0].maps, h[0].args)
                 : ntw == 2 ? launch_cfg<MODE_PRED, 2>(c, h[0].maps, h[0].args)
                            : launch_cfg<MODE_PRED, 1>(c, h[0].maps, h[0].args);
        }
        if (rc) return rc;
        {
            ProfScope p(c, TWA_PROF_CORRECT, mp->w_flops, mp->w_alg);
            rc = ntw == 3   ? launch_cfg<MODE_CORR, 3>(c, h[1].maps, h[1].args)
                 : ntw == 2 ? launch_cfg<MODE_CORR, 2>(c, h[1].maps, h[1].args)
                            : launch_cfg<MODE_CORR, 1>(c, h[1].maps, h[1].args);
        }
        if (rc) return rc;
    } else {
        // the noise of step t + 2 (read by the L.eta tiles of step t + 1) into the
        // buffers of t's parity, which step t's launches do not read. By default
        // the epilogue threads of the two MIX launches draw it between their
        // tiles (half in each launch; the BF16 precisions, whose noise operand is
        // one image), where they would otherwise wait for the next accumulator;
        // else as its own kernel: on a second stream beside the launches (joined
        // before the closing kernel advances the step counter the draw reads), or
        // before them on this stream when profiling
        const bool epi = ts->noise_epi && !ts->Elo && ts->kc != 2;
        const bool side = !epi && ts->overlap_noise && !c->profiling;
        if (side) {
            if ((rc = side_stream(c))) return rc;
            TWA_CUDA(c, cudaEventRecord(ts->ev_fork, c->stream));
            TWA_CUDA(c, cudaStreamWaitEvent(ts->side, ts->ev_fork, 0));
        }
        if (!epi) {
            ProfScope p(c, TWA_PROF_NOISE);
            k_noise_tc<<<nblk(M * (N + 1), 256), 256, 0, side ? ts->side : c->stream>>>(
                ts->E, ts->Elo, ts->XI, ts->E1, ts->Elo1, ts->XI1, M, N, ts->ldk, c->seed, c->d_t, 2,
                c->opts.traj_offset, ts->kc == 2);
        }
        if (side) TWA_CUDA(c, cudaEventRecord(ts->ev_join, ts->side));
        const TcMaps none{};
        TcArgs fa = base_args(c);   // flags of the launch, and the noise draws it carries
        if (epi) {
            fa.nz_E0 = ts->E;
            fa.nz_E1 = ts->E1;
            fa.nz_XI0 = ts->XI;
            fa.nz_XI1 = ts->XI1;
            fa.nz_dt = c->d_t;
            fa.nz_toff = 2;
            fa.nz_m0 = c->opts.traj_offset;
            fa.nz_seed = c->seed;
        }
        const int64_t nz_total = M * (N + 1);
        const GroupDesc* dp = mp->desc + mp->nprob * (t & 1);
        for (int L = 0; L < 2; ++L) {
            const Group g{dp, mp->start, mp->nprob, mp->list[L], mp->first[L], mp->ctas[L]};
            fa.nz_lo = L == 0 ? 0 : nz_total / 2;
            fa.nz_hi = L == 0 ? nz_total / 2 : nz_total;
            ProfScope p(c, L == 0 ? TWA_PROF_PREDICT : TWA_PROF_CORRECT, mp->flops[L], mp->alg[L]);
            rc = ntw == 3   ? launch_cfg<MODE_MIX, 3>(c, none, fa, g, mp->tiles[L])
                 : ntw == 2 ? launch_cfg<MODE_MIX, 2>(c, none, fa, g, mp->tiles[L])
                            : launch_cfg<MODE_MIX, 1>(c, none, fa, g, mp->tiles[L]);
            if (rc) return rc;
        }
        if (side) TWA_CUDA(c, cudaStreamWaitEvent(c->stream, ts->ev_join, 0));
    }
    {
        ProfScope p(c, TWA_PROF_CLOSE);
        k_close_tc<<<nblk(32 * M, 256), 256, 0, c->stream>>>(ts->part, M, ts->n_rt, c->mom, c->d_t, c->n_window,
                                                             c->n_stride, c->d_count, c->d_flags);
    }
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

// Steps t0 .. t0 + steps - 1, launched directly.
int tc_run(twa_ctx* c, int64_t t0, int64_t steps) {
    for (int64_t s = 0; s < steps; ++s) {
        int rc;
        if ((rc = tc_prime(c, t0 + s))) return rc;
        if ((rc = tc_launch_step(c, t0 + s))) return rc;
        tc_steps_done(c, t0 + s + 1);
    }
    return TWA_OK;
}

int tc_get_state(twa_ctx* c, double* sx, double* sy, double* sz) {
    TcState* t = c->tc;
    const int64_t MN = c->M * c->N;
    k_f32_to_f64_rows<<<nblk(MN, 256), 256, 0, c->stream>>>(t->X, t->Y, t->Z, sx, sy, sz, MN);
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

int tc_set_state(twa_ctx* c, const double* sx, const double* sy, const double* sz) {
    TcState* t = c->tc;
    const int64_t MN = c->M * c->N;
    k_f64_to_f32_rows<<<nblk(MN, 256), 256, 0, c->stream>>>(sx, sy, sz, t->X, t->Y, t->Z, MN);
    TWA_CUDA(c, cudaGetLastError());
    return tc_state_changed(c);
}

int tc_field(twa_ctx* c, const double* s, double* P, int64_t K, int which) {
    if (c->fft && which == 0) return fft_field(c, s, P, K);
    TcState* t = c->tc;
    // W: the state's images (hi + lo in the split precisions) and the context's
    // term count. L: the operand rounded once, as the step rounds its noise eta,
    // against L hi + lo in the split precisions (two products; three in the FP32
    // mode, whose eta keeps a lo image) -- the step's L.eta arithmetic.
    const int nterms = which == 1 ? leta_terms(t) : t->terms;
    const bool b_lo = nterms == 3;   // the operand's lo image is read by three-product tiles only
    const int64_t N = c->N, ldk = t->ldk;
    __nv_bfloat16 *hi = nullptr, *lo = nullptr;
    float* out = nullptr;
    const bool tf32 = t->kc == 2;   // FP32 containers; no lo image in the TF32 mode
    const bool with_lo = !(tf32 && t->terms == 1);
    const size_t ni = (size_t)(tf32 ? 4 : 2) * K * ldk;
    // scratch of this call, released (stream-ordered) on every exit below
    auto run = [&]() -> int {
        TWA_CUDA(c, dev_malloc_async(c, &hi, ni, c->stream));
        if (with_lo) TWA_CUDA(c, dev_malloc_async(c, &lo, ni, c->stream));
        TWA_CUDA(c, dev_malloc_async(c, &out, sizeof(float) * K * N, c->stream));
        TWA_CUDA(c, cudaMemsetAsync(hi, 0, ni, c->stream));
        if (with_lo) TWA_CUDA(c, cudaMemsetAsync(lo, 0, ni, c->stream));
        k_split_vectors<<<nblk(K * N, 256), 256, 0, c->stream>>>(s, K, N, ldk, hi, lo, tf32);
        TcMaps fm{};
        fm.a0 = which == 1 ? t->tmLhi : t->tmWhi;
        fm.a1 = which == 1 ? t->tmLlo : t->tmWlo;
        int rc;
        if ((rc = make_map(c, &fm.b0, hi, K, N, ldk, b_box(t), t->kc))) return rc;
        if ((rc = make_map(c, &fm.b1, (with_lo && b_lo) ? lo : hi, K, N, ldk, b_box(t), t->kc))) return rc;
        TcArgs fa = base_args(c);
        fa.n_vec = K;
        fa.field_out = out;
        fa.fsc = (float)(which == 1 ? t->lsc : t->wsc);
        rc = nterms == 3   ? launch_cfg<MODE_FIELD, 3>(c, fm, fa)
             : nterms == 2 ? launch_cfg<MODE_FIELD, 2>(c, fm, fa)
                           : launch_cfg<MODE_FIELD, 1>(c, fm, fa);
        if (rc) return rc;
        k_widen<<<nblk(K * N, 256), 256, 0, c->stream>>>(out, P, K * N);
        TWA_CUDA(c, cudaGetLastError());
        return TWA_OK;
    };
    const int rc = run();
    dev_free_async(c, hi, c->stream);
    dev_free_async(c, lo, c->stream);
    dev_free_async(c, out, c->stream);
    return rc;
}

// ---------------------------------------------------------------------------
// batches: several contexts advanced together, one launch per kernel class

struct TcBatch {
    int n = 0;
    int terms = 3, lterms = 2;   // products per entry of W and of L
    int64_t noise_elems = 0, traj = 0;
    MixPlan* mix = nullptr;   // the mixed launches of all problems
    StepDesc* sd = nullptr;
    int64_t *nstart = nullptr, *mstart = nullptr;
    TcArgs flag_args{};
    twa_ctx* owner = nullptr;   // whose allocator the tables came from
};

void tc_batch_free(TcBatch* b) {
    if (!b) return;
    mix_plan_free(b->mix);
    void* p[] = {b->sd, b->nstart, b->mstart};
    for (void* q : p) dev_free(b->owner, q);
    delete b;
}

int tc_batch_build(twa_ctx* const* ctxs, int n, twa_ctx* lead, TcBatch** out) {
    *out = nullptr;
    TcBatch* b = new TcBatch();
    b->owner = lead;
    b->n = n;
    b->terms = lead->tc->terms;
    b->lterms = lead->tc->lterms;
    std::vector<StepDesc> sd(n);
    std::vector<int64_t> ns(n + 1, 0), ms(n + 1, 0);
    for (int p = 0; p < n; ++p) {
        twa_ctx* c = ctxs[p];
        TcState* t = c->tc;
        if (!t || t->terms != lead->tc->terms || t->lterms != lead->tc->lterms || t->bn != lead->tc->bn ||
            t->kc != lead->tc->kc || t->pair != lead->tc->pair || c->M == 0) {
            tc_batch_free(b);
            return set_error(lead, TWA_EINVAL, "batch: contexts differ in precision or tiles, or have no trajectories");
        }
        t->bn_ready = -1;   // the batch writes the noise-part buffers of its contexts
        sd[p] = StepDesc{t->E, t->E1, t->XI, t->XI1, t->part, c->mom, c->d_t, c->d_count, c->M, c->N, t->ldk,
                         t->n_rt, c->n_window, c->n_stride, c->opts.traj_offset, c->seed};
        ns[p + 1] = ns[p] + c->M * (c->N + 1);
        ms[p + 1] = ms[p] + c->M;
    }
    b->noise_elems = ns[n];
    b->traj = ms[n];
    b->flag_args = base_args(lead);
    b->mix = new MixPlan();
    int rc = mix_plan_build(ctxs, n, lead, b->mix);
    if (rc) {
        tc_batch_free(b);
        return rc;
    }
    bool ok = dev_malloc(lead, &b->sd, sizeof(StepDesc) * n) == cudaSuccess &&
              dev_malloc(lead, &b->nstart, sizeof(int64_t) * (n + 1)) == cudaSuccess &&
              dev_malloc(lead, &b->mstart, sizeof(int64_t) * (n + 1)) == cudaSuccess;
    ok = ok && cudaMemcpy(b->sd, sd.data(), sizeof(StepDesc) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->nstart, ns.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->mstart, ms.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        tc_batch_free(b);
        return set_error(lead, TWA_ENOMEM, "batch: descriptor upload failed");
    }
    *out = b;
    return TWA_OK;
}

// Noise of step t and its noise part for every problem (one grouped L.eta
// launch), into the buffers of t's parity, and the noise of step t + 1: the
// first step of a batch.
int tc_batch_prime(twa_ctx* lead, TcBatch* b, int64_t t) {
    MixPlan* mp = b->mix;
    const int n = b->n;
    k_noise_group<<<nblk(b->noise_elems, 256), 256, 0, lead->stream>>>(b->sd, b->nstart, n, 0);
    // the L.eta descriptors of the other parity write the buffers of t's parity
    const GroupDesc* ld = mp->desc + mp->nprob * ((t & 1) ^ 1) + 2 * n;
    const TcMaps none{};
    const Group g{ld, mp->lstart, n};
    const int rc = b->lterms == 2 ? launch_cfg<MODE_LETA, 2>(lead, none, b->flag_args, g, mp->leta_tiles)
                                  : launch_cfg<MODE_LETA, 1>(lead, none, b->flag_args, g, mp->leta_tiles);
    if (rc) return rc;
    // the noise of step t + 1, read by the L.eta tiles of step t
    k_noise_group<<<nblk(b->noise_elems, 256), 256, 0, lead->stream>>>(b->sd, b->nstart, n, 1);
    TWA_CUDA(lead, cudaGetLastError());
    return TWA_OK;
}

// Step t of every problem (its noise part and the noise of step t + 1 already in
// place): noise of step t + 2, the two mixed launches, window moments, counters.
int tc_batch_step(twa_ctx* lead, TcBatch* b, int64_t t) {
    MixPlan* mp = b->mix;
    const TcMaps none{};
    // as in the single-context step: the draw of step t + 2 on the lead's second
    // stream beside the two launches, joined before the counters advance
    int rc = TWA_OK;
    TcState* lt = lead->tc;
    const bool side = lt->overlap_noise;
    if (side) {
        if ((rc = side_stream(lead))) return rc;
        TWA_CUDA(lead, cudaEventRecord(lt->ev_fork, lead->stream));
        TWA_CUDA(lead, cudaStreamWaitEvent(lt->side, lt->ev_fork, 0));
    }
    k_noise_group<<<nblk(b->noise_elems, 256), 256, 0, side ? lt->side : lead->stream>>>(b->sd, b->nstart, b->n, 2);
    if (side) TWA_CUDA(lead, cudaEventRecord(lt->ev_join, lt->side));
    const GroupDesc* dp = mp->desc + mp->nprob * (t & 1);
    for (int L = 0; L < 2; ++L) {
        const Group g{dp, mp->start, mp->nprob, mp->list[L], mp->first[L], mp->ctas[L]};
        rc = b->terms == 3   ? launch_cfg<MODE_MIX, 3>(lead, none, b->flag_args, g, mp->tiles[L])
             : b->terms == 2 ? launch_cfg<MODE_MIX, 2>(lead, none, b->flag_args, g, mp->tiles[L])
                             : launch_cfg<MODE_MIX, 1>(lead, none, b->flag_args, g, mp->tiles[L]);
        if (rc) return rc;
    }
    if (side) TWA_CUDA(lead, cudaStreamWaitEvent(lead->stream, lt->ev_join, 0));
    k_close_group<<<nblk(32 * b->traj, 256), 256, 0, lead->stream>>>(b->sd, b->mstart, b->n);
    k_advance_group<<<nblk(b->n, 128), 128, 0, lead->stream>>>(b->sd, b->n);
    TWA_CUDA(lead, cudaGetLastError());
    return TWA_OK;
}

int wait_probe(twa_ctx* c, int64_t limit_ns) {
    k_wait_probe<<<1, 32, 0, c->stream>>>(c->d_flags, (unsigned long long)limit_ns);
    TWA_CUDA(c, cudaGetLastError());
    return TWA_OK;
}

// Change the tile configuration of a context (re-encodes its tensor maps).
int tc_set_tiles(twa_ctx* c, int bn, int kc) {
    TcState* t = c->tc;
    mix_free(t);   // its descriptors and the captured steps hold the old tensor maps
    for (auto& g : c->step_graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    t->bn = bn;
    t->kc = kc;
    t->pair = env_int("TWA_TC_PAIR", pair_capable(t) ? 1 : 0) != 0;
    int rc = pair_check(c);
    if (rc) return rc;
    rc = make_matrix_maps(c);
    if (rc) return rc;
    return c->M ? make_state_maps(c) : TWA_OK;
}

}  // namespace twa

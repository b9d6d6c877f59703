// gd_asm_tc.cu -- mixed-precision element kernel whose ICNN layer-2 contractions run
// on the fifth-generation tensor cores (tcgen05.mma, kind::f16 with BF16 operands and
// FP32 accumulation in tensor memory).
//
// A CTA of four warps owns 128 quadrature points at a time (lane = point; warp w holds
// points 32w..32w+31, which are also the tensor-memory lanes that warp may read).  For
// every point the second layer of a network is a dense contraction over the first
// layer's units, and the columns that the forward tangents need form, over the 128
// points, a matrix product
//     D[p][k] = sum_j Z[p][j] W2[k][j],   p = point, k = output unit, j = input unit,
// with M = 128 points, N = K = the network width (padded to 16):
//   energy network (Sec. 4.2 Eq. (dd_0)): Z = s1 (layer-1 softplus) for the value and
//     Z = sg1 * W1[:, c] (c = 0..2) for the three gradient columns (forward tangents),
//     then one reverse column v = W2^T (w3 o sg2) for the Hessian's layer-1 term;
//   yield network (Eq. (Gq_NN)): Z = s1 and Z = sg1 * V1 for G(q) and G'(q), every
//     iteration of the local damage solve (Sec. 3.2 Eq. (dd_7_no_nn)), the 128 points
//     iterating in lockstep with masks.
// Z is written by the threads into shared memory in the canonical no-swizzle K-major
// layout (8 x 16-byte core matrices); the weight tiles are staged once per CTA with a
// bulk asynchronous copy (cp.async.bulk) from a device blob built per handle.  One
// thread issues the MMAs and commits them to an mbarrier; every thread then reads its
// own point's row of D from tensor memory (tcgen05.ld 32x32b) and applies the
// softplus/sigmoid epilogue in FP32.
//
// Operand precision (gd_options.icnn_mma): BF16 (Z and W rounded to 8-bit mantissas,
// FP32 accumulation), or BF16x3 (each operand split into a BF16 high part and a BF16
// residual, three products hi*hi + hi*lo + lo*hi accumulated in FP32: about 16
// significant bits).  Everything else is FP32 element math as in the CUDA-core mixed
// kernel (gd_elem32.cuh); the loading/unloading decision, the history and the residual
// accumulation are FP64.
//
// Paper passages: Sec. 3.1f (kinematics, residual), Sec. 2.2f and Sec. 3.2f Eq.
// (dd_7_no_nn) (local update, KKT), Sec. 3.2f (monolithic tangent), Sec. 4.1f, Sec. 4.2f
// Eqs. (dd_0), (dd_1), (Gq_NN), (dd_7).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gd_elem32.cuh"

namespace gd {
namespace {

using namespace e32;

constexpr int kTcThreads = 128;          // 4 warps = 128 points = 128 tensor-memory lanes
constexpr long long kWaitCycles = 4000000000LL;   // bounded mbarrier waits (about 2 s)

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
// waits for the phase with the given parity to complete; false after kWaitCycles
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(saddr(b)), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}
// bulk asynchronous copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(b))
                 : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// shared-memory matrix descriptor: canonical K-major layout without swizzle, core
// matrices of 8 rows x 16 bytes; lbo = byte step between core matrices along K,
// sbo = byte step between 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                     d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(b))
                 : "memory");
}
// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- operand packing
__device__ __forceinline__ uint32_t bf2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);      // a in the low half (the lower address)
    return *reinterpret_cast<uint32_t *>(&h);
}
// residuals v - bf16(v) of a pair
__device__ __forceinline__ uint32_t bf2_lo(float a, float b)
{
    const float ah = __bfloat162float(__float2bfloat16_rn(a)), bh = __bfloat162float(__float2bfloat16_rn(b));
    return bf2(a - ah, b - bh);
}
// byte offset of (row, 8-element group k8) in a K-major tile with wp columns
__device__ __forceinline__ uint32_t tile_off(int row, int k8, int wp)
{
    return (uint32_t)((row >> 3) * (16 * wp) + k8 * 128 + (row & 7) * 16);
}
__device__ __forceinline__ void st_row8(uint8_t *tile, int row, int k8, int wp, const float (&v)[8])
{
    uint4 u = make_uint4(bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
    *reinterpret_cast<uint4 *>(tile + tile_off(row, k8, wp)) = u;
}
__device__ __forceinline__ void st_row8_lo(uint8_t *tile, int row, int k8, int wp, const float (&v)[8])
{
    uint4 u = make_uint4(bf2_lo(v[0], v[1]), bf2_lo(v[2], v[3]), bf2_lo(v[4], v[5]), bf2_lo(v[6], v[7]));
    *reinterpret_cast<uint4 *>(tile + tile_off(row, k8, wp)) = u;
}

// softplus and sigmoid from one exponential (approximate intrinsics: their error is far
// below the BF16 operand rounding)
__device__ __forceinline__ void sp_sig_fast(float v, float &sp, float &sg)
{
    const float e = __expf(-fabsf(v));
    const float t = 1.0f + e;
    sp = fmaxf(v, 0.0f) + __logf(t);
    const float r = __fdividef(1.0f, t);
    sg = v >= 0.0f ? r : e * r;
}

// D (tmem column d) = A tile x B tile over K = wp (wp / 16 instructions)
__device__ __forceinline__ void mma_tile(uint32_t d, uint32_t a, uint32_t b, int wp, uint32_t acc0)
{
    const uint32_t sbo = 16u * (uint32_t)wp, idesc = idesc_bf16(wp);
    for (int s = 0; s < wp / 16; ++s)
        mma_f16(d, sdesc(a + 256u * s, 128u, sbo), sdesc(b + 256u * s, 128u, sbo), idesc, (s > 0 || acc0) ? 1u : 0u);
}
// one product with the operands in one or two parts: plain D = A B; split D = Ahi Bhi +
// Ahi Blo + Alo Bhi (A's parts in tiles a_hi, a_lo; B's parts at b_hi, b_hi + tile bytes)
template <bool SPLIT>
__device__ __forceinline__ void mma_product(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, int wp)
{
    mma_tile(d, a_hi, b_hi, wp, 0);
    if (SPLIT) {
        const uint32_t b_lo = b_hi + 2u * (uint32_t)(wp * wp);
        mma_tile(d, a_hi, b_lo, wp, 1);
        mma_tile(d, a_lo, b_hi, wp, 1);
    }
}

struct Shared {
    uint8_t *blob, *tiles;
    uint64_t *bar;                       // [0] weight copy, [1] MMA completion, [2] weight slot
    uint32_t tbase;
    uint32_t phase;                      // parity of the next MMA completion to wait for
    uint32_t slot_phase;                 // parity of the next slot copy to wait for
    bool slot_pending;                   // a slot copy was issued and not yet waited for
    bool ok;
};

// every thread waits for the next MMA completion (each commit is waited for by all)
__device__ __forceinline__ void wait_mma(Shared &S, const TcArgs &T)
{
    if (!mbar_wait(S.bar + 1, S.phase)) {
        S.ok = false;
        atomicOr(T.status, 1);
    }
    S.phase ^= 1u;
}

// The weight slot: with both networks on the tensor cores, W2^T (the energy network's
// reverse product) and V2 (the yield network) take turns in one region of shared memory,
// refilled from the L2-resident blob by a bulk copy per batch of 128 points (32 KB per
// batch at width 64, split operands), which lets two CTAs share an SM.
// Every thread calls these at the same program point (CTA-uniform).
__device__ __forceinline__ void slot_wait(Shared &S, const TcArgs &T)
{
    if (!S.slot_pending) return;
    if (!mbar_wait(S.bar + 2, S.slot_phase)) {
        S.ok = false;
        atomicOr(T.status, 1);
    }
    S.slot_phase ^= 1u;
    S.slot_pending = false;
}
// issue the copy of `bytes` from the global blob at `src_off` into the slot (thread 0);
// the slot must be free: no product reading it in flight, no copy pending
__device__ __forceinline__ void slot_fill(Shared &S, const TcArgs &T, int src_off, int bytes, int tid)
{
    if (tid == 0) {
        mbar_expect_tx(S.bar + 2, (uint32_t)bytes);
        bulk_g2s(S.blob + T.s_slot, T.blob + src_off, (uint32_t)bytes, S.bar + 2);
    }
    S.slot_pending = true;
}

// ---------------------------------------------------------------- energy network
// Layer 1 of the energy network for this thread's point; writes the operand rows of
// one round.  Plain: round 0 = (s1, sg1 W1[:,0]), round 1 = (sg1 W1[:,1], sg1 W1[:,2])
// into tiles 0 and 1; split: round r = column r (r = 0: s1, r = 1..3: sg1 W1[:,r-1]),
// high part into tile 0 and residual into tile 1.
template <bool SPLIT>
__device__ __forceinline__ void energy_l1(const float *e32, int w, int wp, const float (&y)[3], int round, uint8_t *t0,
                                          uint8_t *t1, int row)
{
    const float *W1 = e32, *b1 = e32 + 3 * w;
    for (int j8 = 0; j8 < wp / 8; ++j8) {
        float a[8], b[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int j = j8 * 8 + jj;
            float va = 0.0f, vb = 0.0f;
            if (j < w) {
                const float w0 = W1[3 * j], w1 = W1[3 * j + 1], w2 = W1[3 * j + 2];
                const float h = b1[j] + w0 * y[0] + w1 * y[1] + w2 * y[2];
                float sp, sg;
                sp_sig_fast(h, sp, sg);
                if (!SPLIT) {
                    va = round == 0 ? sp : sg * w1;
                    vb = round == 0 ? sg * w0 : sg * w2;
                } else {
                    va = round == 0 ? sp : sg * (round == 1 ? w0 : round == 2 ? w1 : w2);
                }
            }
            a[jj] = va;
            b[jj] = vb;
        }
        st_row8(t0, row, j8, wp, a);
        if (SPLIT) st_row8_lo(t1, row, j8, wp, a);
        else st_row8(t1, row, j8, wp, b);
    }
}

// Value, gradient and Hessian (sym6 order) of the energy network at y for every point
// of the CTA (out10, as psi_net_unit of the CUDA-core kernel):
//   d2N/dy2 = sum_k w3_k sp''(h2_k) g_k g_k^T + sum_j v_j sp''(h1_j) W1_j W1_j^T,
//   v = W2^T (w3 o sp'(h2)).
// CTA-uniform control flow; returns with the tensor memory free for the next product.
template <bool SPLIT>
__device__ void energy_net_tc(Shared &S, const TcArgs &T, const float (&y)[3], float (&out)[10], int tid, int warp)
{
    const TcLayout &L = T.L;
    const int w = L.we, wp = L.wpe;
    const float *e32 = reinterpret_cast<const float *>(S.blob + T.s_e32);
    const float *W1 = e32, *b1 = e32 + 3 * w, *A2 = e32 + 4 * w, *b2 = e32 + 7 * w, *w3 = e32 + 8 * w,
                *a3 = e32 + 9 * w;
    uint8_t *t0 = S.tiles, *t1 = S.tiles + T.tile_bytes;
    const uint32_t a0 = saddr(t0), a1 = saddr(t1), bw = saddr(S.blob), br = saddr(S.blob + T.s_slot);
    const uint32_t lane_base = S.tbase + ((uint32_t)(warp * 32) << 16);
    constexpr int ROUNDS = SPLIT ? 4 : 2;
    // ---- forward columns: type t lands in tensor-memory columns [t wp, (t+1) wp)
    for (int r = 0; r < ROUNDS; ++r) {
        if (r > 0) wait_mma(S, T);           // the previous round's product has read the tiles
        energy_l1<SPLIT>(e32, w, wp, y, r, t0, t1, tid);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_after();
            if (SPLIT) {
                mma_product<true>(S.tbase + (uint32_t)(r * wp), a0, a1, bw, wp);
            } else {
                mma_product<false>(S.tbase + (uint32_t)((2 * r) * wp), a0, a0, bw, wp);
                mma_product<false>(S.tbase + (uint32_t)((2 * r + 1) * wp), a1, a1, bw, wp);
            }
            mma_commit(S.bar + 1);
        }
    }
    wait_mma(S, T);
    tc_after();
    float acc[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[c] = 0.0f;
    for (int k0 = 0; k0 < wp; k0 += 16) {
        float hS[16], g0[16], g1[16], g2[16];
        tmem_ld16(lane_base + (uint32_t)k0, hS);
        tmem_ld16(lane_base + (uint32_t)(wp + k0), g0);
        tmem_ld16(lane_base + (uint32_t)(2 * wp + k0), g1);
        tmem_ld16(lane_base + (uint32_t)(3 * wp + k0), g2);
        tmem_wait_ld();
        float u[16];
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const int k = k0 + kk;
            u[kk] = 0.0f;
            if (k < w) {
                const float c0 = A2[3 * k], c1 = A2[3 * k + 1], c2 = A2[3 * k + 2];
                const float h = hS[kk] + b2[k] + c0 * y[0] + c1 * y[1] + c2 * y[2];
                const float ga = g0[kk] + c0, gb = g1[kk] + c1, gc = g2[kk] + c2;
                float spv, sg;
                sp_sig_fast(h, spv, sg);
                const float wk = w3[k];
                const float e2 = wk * sg * (1.0f - sg);
                acc[0] += wk * spv;
                acc[1] += wk * sg * ga;
                acc[2] += wk * sg * gb;
                acc[3] += wk * sg * gc;
                acc[4] += e2 * ga * ga;
                acc[5] += e2 * ga * gb;
                acc[6] += e2 * ga * gc;
                acc[7] += e2 * gb * gb;
                acc[8] += e2 * gb * gc;
                acc[9] += e2 * gc * gc;
                u[kk] = wk * sg;
            }
        }
        // reverse operand u = w3 o sg2 (the tiles are free: the last forward product is done)
#pragma unroll
        for (int h8 = 0; h8 < 2; ++h8) {
            float v8[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v8[i] = u[h8 * 8 + i];
            st_row8(t0, tid, k0 / 8 + h8, wp, v8);
            if (SPLIT) st_row8_lo(t1, tid, k0 / 8 + h8, wp, v8);
        }
    }
    // ---- reverse column v = W2^T u into columns [0, wp) (W2^T in the weight slot)
    slot_wait(S, T);
    tc_before();
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
        tc_after();
        mma_product<SPLIT>(S.tbase, a0, a1, br, wp);
        mma_commit(S.bar + 1);
    }
    wait_mma(S, T);
    tc_after();
    // the reverse product has read W2^T: the yield network's V2 takes the slot
    if (T.slot_mode == 3) slot_fill(S, T, L.off_v2f, T.v2_bytes, tid);
    for (int j0 = 0; j0 < wp; j0 += 16) {
        float v[16];
        tmem_ld16(lane_base + (uint32_t)j0, v);
        tmem_wait_ld();
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const int j = j0 + jj;
            if (j < w) {
                const float w0 = W1[3 * j], w1 = W1[3 * j + 1], w2 = W1[3 * j + 2];
                const float h = b1[j] + w0 * y[0] + w1 * y[1] + w2 * y[2];
                float spv, sg;
                sp_sig_fast(h, spv, sg);
                const float c = v[jj] * sg * (1.0f - sg);
                acc[4] += c * w0 * w0;
                acc[5] += c * w0 * w1;
                acc[6] += c * w0 * w2;
                acc[7] += c * w1 * w1;
                acc[8] += c * w1 * w2;
                acc[9] += c * w2 * w2;
            }
        }
    }
    tc_before();
#pragma unroll
    for (int c = 0; c < 10; ++c) out[c] = acc[c];
    out[0] += a3[0] * y[0] + a3[1] * y[1] + a3[2] * y[2];
    out[1] += a3[0];
    out[2] += a3[1];
    out[3] += a3[2];
}

// ---------------------------------------------------------------- yield network
// Layer 1 of the yield network at q: s1 = sp(V1 q + c1) and sg1 V1.  Plain: both into
// tiles 0 and 1; split: round 0 = s1, round 1 = sg1 V1 (high part into tile 0,
// residual into tile 1).
template <bool SPLIT>
__device__ __forceinline__ void yield_l1(const float *y32, int w, int wp, float q, int round, uint8_t *t0, uint8_t *t1,
                                         int row)
{
    const float *V1 = y32, *c1 = y32 + w;
    for (int j8 = 0; j8 < wp / 8; ++j8) {
        float a[8], b[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int j = j8 * 8 + jj;
            float va = 0.0f, vb = 0.0f;
            if (j < w) {
                const float v1 = V1[j];
                float sp, sg;
                sp_sig_fast(c1[j] + v1 * q, sp, sg);
                if (!SPLIT) {
                    va = sp;
                    vb = sg * v1;
                } else {
                    va = round == 0 ? sp : sg * v1;
                }
            }
            a[jj] = va;
            b[jj] = vb;
        }
        st_row8(t0, row, j8, wp, a);
        if (SPLIT) st_row8_lo(t1, row, j8, wp, a);
        else st_row8(t1, row, j8, wp, b);
    }
}

// G(q) = s (N_k(q) - N_k(0)) and G'(q) for the points with `need` (CTA-uniform call;
// the yield network has width > 0).
template <bool SPLIT>
__device__ void yield_tc(Shared &S, const TcArgs &T, const NcF &nc, float q, bool need, float &G, float &Gp, int tid,
                         int warp)
{
    const TcLayout &L = T.L;
    const int w = L.wy, wp = L.wpy;
    const float *y32 = reinterpret_cast<const float *>(S.blob + T.s_y32);
    const float *B2 = y32 + 2 * w, *c2 = y32 + 3 * w, *v3 = y32 + 4 * w, *b3 = y32 + 5 * w;
    uint8_t *t0 = S.tiles, *t1 = S.tiles + T.tile_bytes;
    const uint32_t a0 = saddr(t0), a1 = saddr(t1), bv = saddr(S.blob + T.s_slot);
    constexpr int ROUNDS = SPLIT ? 2 : 1;
    slot_wait(S, T);                     // V2 in the weight slot
    for (int r = 0; r < ROUNDS; ++r) {
        if (r > 0) wait_mma(S, T);
        if (need) yield_l1<SPLIT>(y32, w, wp, q, r, t0, t1, tid);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_after();
            if (SPLIT) {
                mma_product<true>(S.tbase + (uint32_t)(r * wp), a0, a1, bv, wp);
            } else {
                mma_product<false>(S.tbase, a0, a0, bv, wp);
                mma_product<false>(S.tbase + (uint32_t)wp, a1, a1, bv, wp);
            }
            mma_commit(S.bar + 1);
        }
    }
    wait_mma(S, T);
    tc_after();
    float n0 = 0.0f, n1 = 0.0f;
    if (__any_sync(0xffffffffu, need)) {
        const uint32_t lane_base = S.tbase + ((uint32_t)(warp * 32) << 16);
        for (int k0 = 0; k0 < wp; k0 += 16) {
            float hS[16], hT[16];
            tmem_ld16(lane_base + (uint32_t)k0, hS);
            tmem_ld16(lane_base + (uint32_t)(wp + k0), hT);
            tmem_wait_ld();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const int k = k0 + kk;
                if (k < w) {
                    const float bk = B2[k];
                    float spv, sg;
                    sp_sig_fast(hS[kk] + c2[k] + bk * q, spv, sg);
                    n0 += v3[k] * spv;
                    n1 += v3[k] * sg * (hT[kk] + bk);
                }
            }
        }
    }
    tc_before();
    G = nc.y_s * (n0 + b3[0] * q - nc.y_N0);
    Gp = nc.y_s * (n1 + b3[0]);
}

// ---------------------------------------------------------------- the kernel
template <int DIM, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads, 1) asm_tc_kernel(AsmArgs A, TcArgs T)
{
    using G_ = Geo<DIM>;
    constexpr int NEN = G_::NEN, NQ = G_::NQ, NDOF = G_::NDOF, EPW = G_::EPW, EPR = G_::EPR;
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    Shared S;
    S.blob = tc_smem;
    S.tiles = tc_smem + T.tiles_off;
    S.bar = reinterpret_cast<uint64_t *>(tc_smem + T.bar_off);
    S.phase = 0;
    S.slot_phase = 0;
    S.slot_pending = false;
    S.ok = true;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(S.bar + 3);
    float *ws = reinterpret_cast<float *>(tc_smem + T.warp_off) + warp * T.warp_floats;
    float *sX = ws;                                  // [EPW][NEN][DIM]
    float *sD = sX + EPW * NEN * DIM;                // [EPW][NEN][NDOF]
    float *sRec = sD + EPW * NEN * NDOF;             // [32][Q_REC]
    float *sVec = reinterpret_cast<float *>(S.tiles) + warp * (EPR * NQ * NEN * V_REC);   // row mode (tiles reused)
    const MatF m = to_f(A.mat);
    const NcF nc = ncf(A.netc[0]);

    if (tid == 0) {
        mbar_init(S.bar, 1);
        mbar_init(S.bar + 1, 1);
        mbar_init(S.bar + 2, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(tslot, (uint32_t)T.ncols);
    tc_before();
    __syncthreads();
    tc_after();
    S.tbase = *tslot;
    // W2, the per-unit vectors and a resident slot (W2^T or V2): bulk copies on one barrier
    if (tid == 0) {
        const int resident = (T.slot_mode == 1 || T.slot_mode == 2) ? T.slot_bytes : 0;
        mbar_expect_tx(S.bar, (uint32_t)(T.fwd_bytes + T.vec_bytes + resident));
        if (T.fwd_bytes > 0) bulk_g2s(S.blob, T.blob + T.L.off_w2f, (uint32_t)T.fwd_bytes, S.bar);
        bulk_g2s(S.blob + T.s_e32, T.blob + T.L.off_e32, (uint32_t)T.vec_bytes, S.bar);
        if (T.slot_mode == 1) bulk_g2s(S.blob + T.s_slot, T.blob + T.L.off_w2r, (uint32_t)T.rev_bytes, S.bar);
        if (T.slot_mode == 2) bulk_g2s(S.blob + T.s_slot, T.blob + T.L.off_v2f, (uint32_t)T.v2_bytes, S.bar);
    }
    if (!mbar_wait(S.bar, 0)) {
        S.ok = false;
        atomicOr(T.status, 1);
    }
    const bool frozen = A.kappa_fixed != nullptr;
    const float tol_r = T.tol_r, tol_br = T.tol_br;

    const int64_t per_cta = 4 * EPW;
    const int64_t n_cb = (A.n_elems + per_cta - 1) / per_cta;
    for (int64_t cb = blockIdx.x; cb < n_cb; cb += gridDim.x) {
        // W2^T into the weight slot for this batch's reverse product: the previous batch's
        // yield products have completed (each was waited for); a V2 copy it never used is
        // consumed first
        if (T.slot_mode == 3) {
            slot_wait(S, T);
            slot_fill(S, T, T.L.off_w2r, T.rev_bytes, tid);
        }
        const int64_t e0 = (cb * 4 + warp) * EPW;
        load_nodes<DIM>(A, e0, sX, sD, lane);
        __syncwarp();
        // ================= qp mode: kinematics and invariants =================
        const int el = lane / NQ, q = lane % NQ;
        const int64_t e_me = e0 + el;
        const bool valid = e_me < A.n_elems;
        float *rec = sRec + lane * Q_REC;
        float F[3][3], H[3][3], phi, g[3], x[3], Jdet;
        qp_kinematics<DIM>(sX, sD, el, q, rec, F, H, phi, g, x, Jdet);
        float Tm[3][3], T2[3][6], y[3];
        input_map(m, x, Jdet, Tm, T2, y);
        // every warp has left the previous batch's row mode (its vectors share the tiles)
        if (__syncthreads_or(!S.ok)) break;
        // ================= energy network (tensor cores) =================
        float o10[10];
        if (m.energy != GD_ENERGY_NEO_HOOKE) energy_net_tc<SPLIT>(S, T, y, o10, tid, warp);
        float ps[3], ph[6], pe;
        energy_derivs(m, nc, x, Jdet, o10, Tm, T2, ps, ph, pe);
        // ================= local damage update, 128 points in lockstep =================
        const float kn = valid ? (float)__ldg(A.kappa_n + e_me * NQ + q) : 0.0f;
        const double kn_d = valid ? __ldg(A.kappa_n + e_me * NQ + q) : 0.0;
        float kappa = kn, Gp = 0.0f, dr = -1.0f, r = 0.0f, lo = kn, hi = kn, dx = 1e30f, dx_prev = 1e30f;
        bool loading = false, fail = false, have_hi = false, took_newton = false;
        int it = 0, n_eval = 0;
        int state = (valid && !frozen) ? 1 : 0;      // 1 trial at kappa_n, 2 warm start, 3 iteration
        if (frozen) kappa = valid ? (float)__ldg(A.kappa_fixed + e_me * NQ + q) : 0.0f;
        for (;;) {
            tc_before();
            if (!__syncthreads_or(state != 0 && S.ok)) break;
            // r(kappa) = G(q(kappa)) - kappa and its slope (Eq. (potential_function)),
            // q = psi_e + qcoef (phi - kappa) / f_d(kappa) (Eq. (ostwald_potential))
            const bool need = state != 0;
            const bool dmg = kappa > m.kappa_d;
            const float f = dmg ? __expf(-m.eta_d * (kappa - m.kappa_d)) : 1.0f;
            const float qv = pe + m.qcoef * (phi - kappa) / f;
            const float dq = m.qcoef * (-1.0f / f + (dmg ? (phi - kappa) * m.eta_d / f : 0.0f));
            float G = qv, Gpv = 1.0f;
            if (T.L.wy > 0) yield_tc<SPLIT>(S, T, nc, qv, need, G, Gpv, tid, warp);
            if (!need) continue;
            ++n_eval;
            Gp = Gpv;
            r = G - kappa;
            dr = Gpv * dq - 1.0f;
            bool step = false;
            if (state == 1) {
                // loading/unloading decided in FP64: Phi_d(kappa_n) = G(q(kappa_n)) - kappa_n > 0
                const double phi_trial = (double)(r + kn) - kn_d;
                if (!(phi_trial > 0.0)) {
                    state = 0;
                    continue;
                }
                loading = true;
                const float kg = A.kappa_guess ? (float)__ldg(A.kappa_guess + e_me * NQ + q) : kn;
                if (kg > kn && isfinite(kg)) {
                    kappa = kg;
                    state = 2;
                    continue;
                }
                lo = kappa;
                step = true;
            } else {
                if (r > 0.0f) {
                    lo = kappa;
                } else {
                    hi = kappa;
                    have_hi = true;
                }
                if (state == 2) {
                    dx_prev = have_hi ? hi - lo : 1.0e30f;
                    dx = dx_prev;
                } else {
                    ++it;
                }
                step = true;
            }
            if (step) {
                // the lazily bracketed, safeguarded Newton iteration of the CUDA-core kernel
                state = 3;
                const float scale = fabsf(kappa) > 1.0f ? fabsf(kappa) : 1.0f;
                if (it >= m.local_max) {
                    fail = true;
                    state = 0;
                } else if (fabsf(r) <= tol_r * scale || (have_hi && (hi - lo) <= tol_br * scale)) {
                    state = 0;
                } else if (fabsf(r) <= 0.1f * tol_r * scale * fabsf(dr) &&
                           (have_hi ? (hi - lo) <= 1e-2f * scale
                                    : (took_newton && fabsf(2.0f * r) <= fabsf(dx * dr)))) {
                    // the next Newton correction is within a tenth of the tolerance, with the
                    // root bracketed within 1e-2 or the iteration converging from one side
                    // (near full damage r' grows like 1 / f_d and |r| stays at its rounding)
                    state = 0;
                } else {
                    const float newton = kappa - r / dr;
                    bool take;
                    if (have_hi) {
                        take = (newton > lo) && (newton < hi) && (fabsf(2.0f * r) <= fabsf(dx_prev * dr));
                    } else {
                        const float cap = 4.0f * ((r > 1e-12f ? r : 1e-12f) + (kappa - kn));
                        take = dr < 0.0f && newton > lo && (newton - kappa) <= cap;
                    }
                    dx_prev = dx;
                    took_newton = take;
                    if (take) {
                        dx = kappa - newton;
                        kappa = newton;
                    } else if (have_hi) {
                        dx = 0.5f * (hi - lo);
                        kappa = lo + dx;
                    } else {
                        const float rr = r > 1e-12f ? r : 1e-12f;
                        const float st = 2.0f * ((kappa - kn) > rr ? (kappa - kn) : rr);
                        dx = st;
                        kappa = lo + st;
                    }
                }
            }
        }
        if (__syncthreads_or(!S.ok)) break;
        // ================= qp mode: history, stress and records =================
        if (valid) {
            atomicAdd(A.counters + 2, n_eval);
            if (A.kappa_new)
                A.kappa_new[e_me * NQ + q] = frozen ? __ldg(A.kappa_fixed + e_me * NQ + q)
                                             : loading ? fmax(kn_d, (double)kappa) : kn_d;
            if (A.loading) A.loading[e_me * NQ + q] = loading ? 1 : 0;
            if (fail) atomicAdd(A.counters, 1);
            if (loading) atomicAdd(A.counters + 1, 1);
        }
        stress_records(m, F, x, g, phi, Jdet, ps, ph, kappa, loading, Gp, dr, valid, rec);
        // every warp is done with the tiles (the last product completed) before the row
        // mode writes its vectors over them
        __syncthreads();
        row_mode<DIM>(A, m, sRec, sVec, e0, lane);
    }
    slot_wait(S, T);                     // no copy into shared memory outlives the CTA
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(S.tbase, (uint32_t)T.ncols);
}

// Canonical tiles and FP32 vectors of the two networks (see TcLayout).
__global__ void tc_blob_kernel(const float *pe, int we, const float *py, int wy, TcLayout L, uint8_t *blob)
{
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    auto put = [&](int off, int wp, int w, const float *W2, bool transpose) {
        const int tile = 2 * wp * wp;
        for (int i = t0; i < wp * wp; i += stride) {
            const int n = i / wp, k = i % wp;
            float v = 0.0f;
            if (n < w && k < w) v = transpose ? W2[k * w + n] : W2[n * w + k];
            const uint32_t o = (uint32_t)((n >> 3) * (16 * wp) + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2);
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            *reinterpret_cast<__nv_bfloat16 *>(blob + off + o) = hi;
            if (L.split) *reinterpret_cast<__nv_bfloat16 *>(blob + off + tile + o) = __float2bfloat16_rn(v - __bfloat162float(hi));
        }
    };
    if (we > 0) {
        const float *W1 = pe, *b1 = W1 + 3 * we, *W2 = b1 + we, *A2 = W2 + we * we, *b2 = A2 + 3 * we,
                    *w3 = b2 + we, *a3 = w3 + we;
        put(L.off_w2f, L.wpe, we, W2, false);
        put(L.off_w2r, L.wpe, we, W2, true);
        float *e = reinterpret_cast<float *>(blob + L.off_e32);
        for (int i = t0; i < 3 * we; i += stride) e[i] = W1[i];
        for (int i = t0; i < we; i += stride) e[3 * we + i] = b1[i];
        for (int i = t0; i < 3 * we; i += stride) e[4 * we + i] = A2[i];
        for (int i = t0; i < we; i += stride) {
            e[7 * we + i] = b2[i];
            e[8 * we + i] = w3[i];
        }
        for (int i = t0; i < 3; i += stride) e[9 * we + i] = a3[i];
    }
    if (wy > 0) {
        const float *V1 = py, *c1 = V1 + wy, *V2 = c1 + wy, *B2 = V2 + wy * wy, *c2 = B2 + wy, *v3 = c2 + wy,
                    *b3 = v3 + wy;
        put(L.off_v2f, L.wpy, wy, V2, false);
        float *f = reinterpret_cast<float *>(blob + L.off_y32);
        for (int i = t0; i < wy; i += stride) {
            f[i] = V1[i];
            f[wy + i] = c1[i];
            f[2 * wy + i] = B2[i];
            f[3 * wy + i] = c2[i];
            f[4 * wy + i] = v3[i];
        }
        if (t0 == 0) f[5 * wy] = b3[0];
    }
}

int round16(int w) { return (w + 15) / 16 * 16; }

}  // namespace

TcLayout tc_layout(int we, int wy, bool split)
{
    TcLayout L{};
    L.we = we;
    L.wy = wy;
    L.wpe = we > 0 ? round16(we) : 0;
    L.wpy = wy > 0 ? round16(wy) : 0;
    L.split = split ? 1 : 0;
    const int parts = split ? 2 : 1;
    int off = 0;
    L.off_w2f = off;
    off += parts * 2 * L.wpe * L.wpe;
    L.off_w2r = off;
    off += parts * 2 * L.wpe * L.wpe;
    L.off_v2f = off;
    off += parts * 2 * L.wpy * L.wpy;
    L.off_e32 = off;
    off += ((9 * we + 3) * 4 + 15) / 16 * 16;
    L.off_y32 = off;
    off += ((5 * wy + 1) * 4 + 15) / 16 * 16;
    L.bytes = off;
    return L;
}

cudaError_t tc_build_blob(const DevNet &psi, const DevNet &yld, const TcLayout &L, uint8_t *blob, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(blob, 0, (size_t)L.bytes, s);
    if (e != cudaSuccess) return e;
    tc_blob_kernel<<<32, 256, 0, s>>>(psi.pf, L.we, yld.pf, L.wy, L, blob);
    return cudaGetLastError();
}

namespace {
template <int DIM, bool SPLIT>
cudaError_t launch_tc_t(const AsmArgs &a, const TcLaunch &c, cudaStream_t s)
{
    using G_ = Geo<DIM>;
    TcArgs T{};
    T.L = c.L;
    T.blob = c.blob;
    T.status = c.status;
    T.tol_r = SPLIT ? 4e-5f : 4e-3f;
    T.tol_br = SPLIT ? 2e-5f : 2e-3f;
    const int wpmax = c.L.wpe > c.L.wpy ? c.L.wpe : c.L.wpy;
    // tensor memory: four energy columns of width wp (or two yield columns), a power of two >= 32
    int need_cols = 4 * c.L.wpe > 2 * c.L.wpy ? 4 * c.L.wpe : 2 * c.L.wpy;
    int ncols = 32;
    while (ncols < need_cols) ncols *= 2;
    T.ncols = ncols;
    // weights in shared memory: W2 | the slot (W2^T and/or V2) | FP32 vectors
    const bool energy_tc = a.mat.energy != GD_ENERGY_NEO_HOOKE && c.L.we > 0;
    const bool yield_tc_on = c.L.wy > 0 && a.kappa_fixed == nullptr;    // frozen history: no local solve
    T.fwd_bytes = energy_tc ? c.L.off_w2r - c.L.off_w2f : 0;
    T.rev_bytes = c.L.off_v2f - c.L.off_w2r;
    T.v2_bytes = c.L.off_e32 - c.L.off_v2f;
    T.vec_bytes = c.L.bytes - c.L.off_e32;
    T.slot_mode = energy_tc ? (yield_tc_on ? 3 : 1) : (yield_tc_on ? 2 : 0);
    T.slot_bytes = T.slot_mode == 3 ? (T.rev_bytes > T.v2_bytes ? T.rev_bytes : T.v2_bytes)
                   : T.slot_mode == 1 ? T.rev_bytes
                   : T.slot_mode == 2 ? T.v2_bytes
                                      : 0;
    T.s_slot = T.fwd_bytes;
    T.s_e32 = T.s_slot + T.slot_bytes;
    T.s_y32 = T.s_e32 + (c.L.off_y32 - c.L.off_e32);
    // shared memory: weights | two operand tiles (also the row-mode vectors) | per-warp scratch | barriers
    size_t off = ((size_t)(T.s_e32 + T.vec_bytes) + 1023) / 1024 * 1024;
    T.tiles_off = (int)off;
    T.tile_bytes = 128 * (wpmax > 0 ? wpmax : 16) * 2;
    const size_t vec_bytes = (size_t)4 * G_::EPR * G_::NQ * G_::NEN * V_REC * sizeof(float);
    size_t tiles = 2 * (size_t)T.tile_bytes;
    if (tiles < vec_bytes) tiles = vec_bytes;
    off += (tiles + 1023) / 1024 * 1024;
    T.warp_off = (int)off;
    T.warp_floats = G_::EPW * G_::NEN * (DIM + G_::NDOF) + 32 * Q_REC;
    off += (size_t)4 * T.warp_floats * sizeof(float);
    off = (off + 15) / 16 * 16;
    T.bar_off = (int)off;
    off += 32;
    size_t smem = off;
    int dev = 0, optin = 0, smem_sm = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // never more resident CTAs per SM than the tensor memory holds (512 columns): pad the
    // shared memory so that one more CTA would not fit
    const int tmem_cap = 512 / ncols;
    const size_t per_cta_min = (size_t)smem_sm / (size_t)(tmem_cap + 1) + 1;
    if (smem < per_cta_min) smem = per_cta_min;
    if (smem > (size_t)optin) return cudaErrorInvalidConfiguration;
    auto fn = asm_tc_kernel<DIM, SPLIT>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // all of the unified L1/shared storage as shared memory: two CTAs of ~108 KB
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM from the shared memory (with the per-block reservation), the
    // registers and the tensor memory; the occupancy query is taken as a lower bound (it
    // has answered 1 where two CTAs fit).  The grid-stride loop is correct for any grid.
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTcThreads, smem);
    if (e != cudaSuccess) return e;
    {
        cudaFuncAttributes fa{};
        int reserved = 0;
        e = cudaFuncGetAttributes(&fa, fn);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e != cudaSuccess) return e;
        const int regs_cta = ((fa.numRegs * 32 + 255) / 256 * 256) * (kTcThreads / 32);
        int fit = (int)((size_t)smem_sm / (smem + (size_t)fa.sharedSizeBytes + (size_t)reserved));
        if (regs_cta > 0 && 65536 / regs_cta < fit) fit = 65536 / regs_cta;
        if (fit > per_sm) per_sm = fit;
    }
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    const int64_t per_cta = 4 * G_::EPW;
    const int64_t n_cb = (a.n_elems + per_cta - 1) / per_cta;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > n_cb) grid = n_cb;
    if (c.grid_max > 0 && grid > c.grid_max) grid = c.grid_max;
    if (grid < 1) grid = 1;
    fn<<<(unsigned)grid, kTcThreads, smem, s>>>(a, T);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_assemble_tc(int dim, const AsmArgs &a, const TcLaunch &c, cudaStream_t s)
{
    if (a.n_elems <= 0) return cudaSuccess;
    if (a.psi_tab || a.yld_tab) return cudaErrorInvalidValue;      // one weight set per launch
    if (dim == 2) return c.L.split ? launch_tc_t<2, true>(a, c, s) : launch_tc_t<2, false>(a, c, s);
    return c.L.split ? launch_tc_t<3, true>(a, c, s) : launch_tc_t<3, false>(a, c, s);
}

}  // namespace gd

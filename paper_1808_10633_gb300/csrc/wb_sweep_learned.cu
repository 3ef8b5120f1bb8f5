// wb_sweep_learned.cu -- FP32 WENO5 sweep with learned nonlinear weights.
//
// The characteristic sweep of wb_sweep.cuh (Sec. 2.1 eq. FWENO) with one
// change: for every interface, field and side, the weights (w0, w2) of phi_N
// come from a small per-field network (6 -> 32 -> 32 -> 3, GELU, softmax)
// evaluated on the normalised split-flux stencil, unless a detector fires
// (a jump in the four differences phi_N reads, or a pressure ratio across the
// six stencil cells), in which case the Jiang-Shu weights are kept.
//
// Network evaluation on the tensor cores: all 32 lanes of a warp reach the
// same field together, so the warp runs the network on a 64 x 6 batch (two
// sides per lane) with mma.sync.m16n8k8 (first layer, the bias folded in as
// a seventh input equal to 1) and mma.sync.m16n8k16 (hidden and output
// layers), BF16 operands and FP32 accumulators.  A layer's accumulator
// fragments are re-packed in registers as the next layer's A fragments; the
// weights are stored already in B-fragment order (34 words per lane per
// field in groups of four, so that a warp reads each group as one 16-byte
// load per lane; written by wb_set_mlp on the host side).  The GELU (sigmoid
// form) takes one hardware tanh and one FMA on BF16 pairs, the constant of
// its argument folded into the stored weights (gelu_k).  Batch rows are
// independent, so a lane whose interface lies outside the patch still joins
// the warp-wide products (with a valid stencil) and only skips its store.
#include "wb_sweep.cuh"

#include <cuda_bf16.h>

namespace wb {
namespace {

#ifndef WB_LEARNED_NT
#define WB_LEARNED_NT 256                        // threads (interfaces) per tile
#endif
#ifndef WB_LEARNED_MINB
#define WB_LEARNED_MINB 2                        // resident blocks per SM (256 threads: 128 registers)
#endif
constexpr int kLearnedNT = WB_LEARNED_NT;
static_assert(kLearnedNT % 32 == 0 && kLearnedNT >= 64 && kLearnedNT <= 512, "learned tile size");
// Tile of the learned sweep: the Jiang-Shu sweep's extent along the axis,
// kLearnedNT / TA pencils.
template <int AXIS>
struct LShape {
    static constexpr int TA = Shape<AXIS>::TA, TP = kLearnedNT / TA;
    static_assert(TA * TP == kLearnedNT, "learned tile size must be a multiple of the tile's axis extent");
};

constexpr int kMlpWords = 36;                    // per lane per field (34 used), 9 groups of 4
// Word k of lane `lane` within one field's fragment table: groups of four
// consecutive words per lane, the 32 lanes' groups side by side, so that a
// warp reads one group of every lane as one coalesced 16-byte load each.
__host__ __device__ constexpr int frag_index(int k, int lane) { return ((k >> 2) * 32 + lane) * 4 + (k & 3); }
constexpr float kGeluK = 0.851f;                 // gelu(x) = x/2 (1 + tanh(kGeluK x))
constexpr int kMlpSmemWords = WB_MLP_NFIELD * kMlpWords * 32;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// The same with the accumulator input C given apart from D (zeros or the
// layer's bias), so D needs no initialisation.
__device__ __forceinline__ void mma_k8_c(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0, float c0, float c1,
                                         float c2, float c3) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%8,%9,%10};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
}

__device__ __forceinline__ void mma_k16_c(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1,
                                          float c0, float c1, float c2, float c3) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
}

__device__ __forceinline__ void mma_k16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The GELU in its sigmoid form, gelu(x) = x sigma(1.702 x) = x/2 (1 +
// tanh(0.851 x)), on two FP32 accumulators, returned as the next layer's BF16
// operand pair.  The host stores every layer's pre-activation scaled by
// k = 0.851 (the first layer's weights and bias and the hidden bias times k,
// the hidden weights halved), so the accumulators hold y = k x and the pair
// y + y tanh(y) = 2 k gelu(x) needs one tanh and one fused multiply-add on
// the packed BF16 pair; the output layer's weights are divided by 2 k.
__device__ __forceinline__ uint32_t gelu_k(float a, float b) {
    const uint32_t y = pack_bf16(a, b);
    uint32_t t, r;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(y));
    asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(r) : "r"(y), "r"(t));                // y + y t
    return r;
}

// One warp, one field: omega (w0, w2) for the 64 rows of `in` (row r holds 8
// bf16: x0..x5, 1, 0) into om[2r], om[2r+1].
#ifndef WB_LEARNED_PACKED
#define WB_LEARNED_PACKED 1            // input normalisation and weights in packed FP32 pairs
#endif
#ifndef WB_LEARNED_HOIST
#define WB_LEARNED_HOIST 0
#endif
// This lane's fragment words of one field: read from shared memory at each
// use, or (WB_LEARNED_HOIST) once into registers for all four row tiles.
struct WordsSmem {
    const uint32_t* W;
    int lane;
    __device__ __forceinline__ uint32_t operator()(int k) const { return W[frag_index(k, lane)]; }
    __device__ __forceinline__ uint4 q(int grp) const { return reinterpret_cast<const uint4*>(W)[grp * 32 + lane]; }
};
struct WordsReg {
    uint32_t w[kMlpWords];
    __device__ __forceinline__ WordsReg(const uint32_t* W, int lane) {
#pragma unroll
        for (int k = 0; k < kMlpWords; k++) w[k] = W[frag_index(k, lane)];
    }
    __device__ __forceinline__ uint32_t operator()(int k) const { return w[k]; }
    __device__ __forceinline__ uint4 q(int grp) const {
        return make_uint4(w[4 * grp], w[4 * grp + 1], w[4 * grp + 2], w[4 * grp + 3]);
    }
};

// K row tiles of 16 starting at tile mt0, their products interleaved (K
// independent chains of MMAs, GELUs and softmaxes for the scheduler).
template <int K, class Words>
__device__ __forceinline__ void mlp_tiles(const Words& W, const uint32_t* __restrict__ in, float* __restrict__ om,
                                          int lane, int mt0) {
    const int g = lane >> 2, t = lane & 3;
    uint32_t a0[K], a1[K];
#pragma unroll
    for (int q = 0; q < K; q++) {
        const int r0 = 16 * (mt0 + q) + g;
        a0[q] = in[r0 * 4 + t];
        a1[q] = in[(r0 + 8) * 4 + t];
    }
    float c1[K][4][4];
    {
        const uint4 w1 = W.q(0);
        const uint32_t b[4] = {w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
            for (int q = 0; q < K; q++) mma_k8_c(c1[q][nt], a0[q], a1[q], b[nt], 0.f, 0.f, 0.f, 0.f);
    }
    uint32_t A2[K][2][4];
#pragma unroll
    for (int q = 0; q < K; q++)
#pragma unroll
        for (int kt = 0; kt < 2; kt++) {
            A2[q][kt][0] = gelu_k(c1[q][2 * kt][0], c1[q][2 * kt][1]);
            A2[q][kt][1] = gelu_k(c1[q][2 * kt][2], c1[q][2 * kt][3]);
            A2[q][kt][2] = gelu_k(c1[q][2 * kt + 1][0], c1[q][2 * kt + 1][1]);
            A2[q][kt][3] = gelu_k(c1[q][2 * kt + 1][2], c1[q][2 * kt + 1][3]);
        }
    float c2[K][4][4];
    {
        const uint4 bb0 = W.q(6), bb1 = W.q(7);      // hidden bias pairs of n tiles 0, 1 and 2, 3
        const uint32_t bias[8] = {bb0.x, bb0.y, bb0.z, bb0.w, bb1.x, bb1.y, bb1.z, bb1.w};
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            const float blo = __uint_as_float(bias[2 * nt]), bhi = __uint_as_float(bias[2 * nt + 1]);
            const uint4 w2 = W.q(1 + nt);
#pragma unroll
            for (int q = 0; q < K; q++) {
                mma_k16_c(c2[q][nt], A2[q][0], w2.x, w2.y, blo, bhi, blo, bhi);
                mma_k16(c2[q][nt], A2[q][1], w2.z, w2.w);
            }
        }
    }
    uint32_t A3[K][2][4];
#pragma unroll
    for (int q = 0; q < K; q++)
#pragma unroll
        for (int kt = 0; kt < 2; kt++) {
            A3[q][kt][0] = gelu_k(c2[q][2 * kt][0], c2[q][2 * kt][1]);
            A3[q][kt][1] = gelu_k(c2[q][2 * kt][2], c2[q][2 * kt][3]);
            A3[q][kt][2] = gelu_k(c2[q][2 * kt + 1][0], c2[q][2 * kt + 1][1]);
            A3[q][kt][3] = gelu_k(c2[q][2 * kt + 1][2], c2[q][2 * kt + 1][3]);
        }
    float c3[K][4];
    {
        const uint4 w3 = W.q(5), b3 = W.q(8);
        const float b3lo = __uint_as_float(b3.x), b3hi = __uint_as_float(b3.y);
#pragma unroll
        for (int q = 0; q < K; q++) {
            mma_k16_c(c3[q], A3[q][0], w3.x, w3.y, b3lo, b3hi, b3lo, b3hi);
            mma_k16(c3[q], A3[q][1], w3.z, w3.w);
        }
    }
#pragma unroll
    for (int q = 0; q < K; q++) {
        const int r0 = 16 * (mt0 + q) + g, r1 = r0 + 8;
        // logits z0, z1 sit in lane t = 0 of each quad, z2 in lane t = 1 (row
        // r0 in c3[0..1], row r1 in c3[2..3]); lane t = 0 takes the softmax
        // of row r0 and lane t = 1 that of row r1
        const float z2a = __shfl_down_sync(0xffffffffu, c3[q][0], 1);
        const float z0b = __shfl_up_sync(0xffffffffu, c3[q][2], 1);
        const float z1b = __shfl_up_sync(0xffffffffu, c3[q][3], 1);
        if (t < 2) {
            const float z0 = t == 0 ? c3[q][0] : z0b, z1 = t == 0 ? c3[q][1] : z1b;
            const float z2 = t == 0 ? z2a : c3[q][2];
            const float zm = fmaxf(z0, fmaxf(z1, z2));
            const float e0 = __expf(z0 - zm), e1 = __expf(z1 - zm), e2 = __expf(z2 - zm);
            const float inv = __fdividef(1.0f, e0 + e1 + e2);
            const int r = t == 0 ? r0 : r1;
            om[2 * r] = e0 * inv;
            om[2 * r + 1] = e2 * inv;
        }
    }
}

// Row tiles evaluated together by one warp (1: one tile at a time).
#ifndef WB_LEARNED_ILP
#define WB_LEARNED_ILP 1
#endif
__device__ __forceinline__ void mlp_warp(const uint32_t* __restrict__ Ws, const uint32_t* __restrict__ in,
                                         float* __restrict__ om, int lane, int ntiles = 4) {
#if WB_LEARNED_HOIST
    const WordsReg W(Ws, lane);
#else
    const WordsSmem W{Ws, lane};
#endif
    int mt = 0;
#if WB_LEARNED_ILP > 1
#pragma unroll 1
    for (; mt + 2 <= ntiles; mt += 2) mlp_tiles<2>(W, in, om, lane, mt);
#endif
#pragma unroll 1
    for (; mt < ntiles; mt++) mlp_tiles<1>(W, in, om, lane, mt);
}

// The learned sweep projects the stencil's differences like the Jiang-Shu
// sweep (parked values in shared memory, the weight fragments then read from
// global memory through L1 instead of a shared copy), or with
// WB_LEARNED_DELTA=0 the stencil's values in two groups of fields.
#ifndef WB_LEARNED_DELTA
#define WB_LEARNED_DELTA 1
#endif

// Weight policy of the learned scheme.
struct LearnedWeights {
    static constexpr bool kDiff = WB_LEARNED_DELTA != 0;
    const uint32_t* W;        // shared, [field][34][32]
    uint32_t* in;             // shared, this warp's 64 x 4 words
    float* om;                // shared, this warp's 64 x 2
    int lane;
    bool pfire;               // pressure detector of this interface
    float kappa;
    float smooth;             // network only where (eps + max IS) > smooth (eps + min IS)
    int nfire = 0;            // Jiang-Shu decisions of this thread (fields x sides)

    // The smoothness gate: true where the smoothness indicators of phi_N's
    // four differences (Sec. 2.1) spread by more than `smooth`.
    __device__ __forceinline__ bool rough(float a, float b, float c, float d) const {
        const float t0 = a - b, t1 = a - 3.0f * b, t2 = b - c, t3 = b + c, t4 = c - d, t5 = 3.0f * c - d;
        const float is0 = 13.0f * t0 * t0 + 3.0f * t1 * t1;
        const float is1 = 13.0f * t2 * t2 + 3.0f * t3 * t3;
        const float is2 = 13.0f * t4 * t4 + 3.0f * t5 * t5;
        const float mx = fmaxf(is0, fmaxf(is1, is2)), mn = fminf(is0, fminf(is1, is2));
        return mx + 1e-6f > smooth * (mn + 1e-6f);
    }

    __device__ __forceinline__ float corr(int s, const float (&w)[6], const float (&g)[6], float alpha) {
#if WB_LEARNED_PACKED
        return corr_packed(s, w, g, alpha);
#endif
        const float ha = 0.5f * alpha;
        float vp[6], vm[6];
#pragma unroll
        for (int k = 0; k < 6; k++) {
            vp[k] = 0.5f * g[k] + ha * w[k];
            vm[k] = 0.5f * g[5 - k] - ha * w[5 - k];     // '-' side reversed
        }
        float Dp[4], Dm[4];
#pragma unroll
        for (int k = 0; k < 4; k++) { Dp[k] = vp[k + 1] - vp[k]; Dm[k] = vm[k] - vm[k + 1]; }
        // Dp = (D+_{i-3/2}, .., D+_{i+3/2}); Dm = (D-_{i+5/2}, .., D-_{i-1/2})
        bool fire[2];
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const float* v = side == 0 ? vp : vm;
            float mean = 0.f;
#pragma unroll
            for (int k = 0; k < 6; k++) mean += v[k];
            mean *= (1.0f / 6.0f);
            float mx = 0.f;
#pragma unroll
            for (int k = 0; k < 6; k++) mx = fmaxf(mx, fabsf(v[k] - mean));
            const float inv = __fdividef(1.0f, mx + 1e-12f);
            const int r = 2 * lane + side;
            // one 16-byte store per row (four 4-byte stores at an 8-word lane
            // stride would meet in 4 banks)
            *reinterpret_cast<uint4*>(in + r * 4) =
                make_uint4(pack_bf16((v[0] - mean) * inv, (v[1] - mean) * inv),
                           pack_bf16((v[2] - mean) * inv, (v[3] - mean) * inv),
                           pack_bf16((v[4] - mean) * inv, (v[5] - mean) * inv), pack_bf16(1.0f, 0.0f));
            const float* D = side == 0 ? Dp : Dm;
            float a[4], dmax = 0.f, dsum = 0.f;
#pragma unroll
            for (int k = 0; k < 4; k++) { a[k] = fabsf(D[k]); dmax = fmaxf(dmax, a[k]); dsum += a[k]; }
            fire[side] = pfire || dmax > kappa * (dsum - dmax) * (1.0f / 3.0f) + 1e-30f
                         || !rough(D[0], D[1], D[2], D[3]);
            nfire += fire[side] ? 1 : 0;
        }
        __syncwarp();
        mlp_warp(W + s * kMlpWords * 32, in, om, lane);
        __syncwarp();
        const float4 wl = *reinterpret_cast<const float4*>(om + 4 * lane);
        const float w0p = wl.x, w2p = wl.y, w0m = wl.z, w2m = wl.w;
        __syncwarp();
        const float php = fire[0] ? phi_n(Dp[0], Dp[1], Dp[2], Dp[3])
                                  : w0p * (Dp[0] - 2.f * Dp[1] + Dp[2]) * (1.f / 3.f)
                                        + (w2p - 0.5f) * (Dp[1] - 2.f * Dp[2] + Dp[3]) * (1.f / 6.f);
        const float phm = fire[1] ? phi_n(Dm[0], Dm[1], Dm[2], Dm[3])
                                  : w0m * (Dm[0] - 2.f * Dm[1] + Dm[2]) * (1.f / 3.f)
                                        + (w2m - 0.5f) * (Dm[1] - 2.f * Dm[2] + Dm[3]) * (1.f / 6.f);
        return phm - php;
    }

    // The same in packed FP32 pairs, lane x the '+' side and lane y the '-'
    // side (its stencil reversed).  The pair differences V_{k+1} - V_k are
    // (D+_k, -D-_k); both the interpolant and the learned form are odd in D,
    // so the '-' side's value is the negative of the one taken on -D-.
    __device__ __forceinline__ float corr_packed(int s, const float (&w)[6], const float (&g)[6], float alpha) {
        const float2 ha = make_float2(0.5f * alpha, -0.5f * alpha);
        float2 V[6];
#pragma unroll
        for (int k = 0; k < 6; k++)
            V[k] = __ffma2_rn(ha, make_float2(w[k], w[5 - k]), __fmul2_rn(splat2(0.5f), make_float2(g[k], g[5 - k])));
        float2 D[4];
#pragma unroll
        for (int k = 0; k < 4; k++) D[k] = __ffma2_rn(V[k], splat2(-1.0f), V[k + 1]);
        return corr_vd(s, V, D);
    }

    // The same from the projected differences dw_m = l (U_{m+1} - U_m), dg_m
    // = l (F_{m+1} - F_m): the split differences are (dg_m +- alpha dw_m)/2,
    // and the split fluxes are their running sums up to a constant, which
    // the network's input normalisation (v - mean v) / max|v - mean v|
    // does not see.
    // The split differences are taken twice over (dg +- alpha dw, the
    // Jiang-Shu sweep's exact scaling): the inputs' normalisation and the
    // detectors do not see the factor, the gate and phi_N take 4 eps, and
    // corr_vd halves its result.
    __device__ __forceinline__ float corr_d(int s, const float (&dw)[5], const float (&dg)[5], float alpha) {
        float dP[5], dM[5];
#pragma unroll
        for (int m = 0; m < 5; m++) {
            dP[m] = fmaf(alpha, dw[m], dg[m]);
            dM[m] = fmaf(-alpha, dw[m], dg[m]);
        }
        float2 D[4], V[6];
        V[0] = splat2(0.0f);
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const float2 d = make_float2(dP[k], -dM[4 - k]);
            if (k < 4) D[k] = d;
            V[k + 1] = __fadd2_rn(V[k], d);
        }
        return corr_vd<true>(s, V, D);
    }

    // Lane x the '+' side, lane y the '-' side with its stencil reversed:
    // V the six split fluxes (up to a constant), D their four differences;
    // TWICE: both taken twice over.
    template <bool TWICE = false>
    __device__ __forceinline__ float corr_vd(int s, const float2 (&V)[6], const float2 (&D)[4]) {
        constexpr float kEps3 = TWICE ? 4.0f * kEps3f : kEps3f;
        bool fire[2];
#pragma unroll
        for (int side = 0; side < 2; side++) {
            float dmax = 0.f, dsum = 0.f;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float a = fabsf(side == 0 ? D[k].x : D[k].y);
                dmax = fmaxf(dmax, a);
                dsum += a;
            }
            fire[side] = pfire || dmax > kappa * (dsum - dmax) * (1.0f / 3.0f) + 1e-30f;
        }
        {
            // smoothness gate on both sides at once (the indicators are even
            // in D, so lane y's negated differences give the '-' side's),
            // compared as (eps + IS_k)/3 like phi_N forms them
            const float2 k13 = splat2(13.0f / 3.0f), eps3 = splat2(kEps3);
            const float2 t0 = __ffma2_rn(D[1], splat2(-1.0f), D[0]), t1 = __ffma2_rn(D[1], splat2(-3.0f), D[0]);
            const float2 t2 = __ffma2_rn(D[2], splat2(-1.0f), D[1]), t3 = __fadd2_rn(D[1], D[2]);
            const float2 t4 = __ffma2_rn(D[3], splat2(-1.0f), D[2]), t5 = __ffma2_rn(D[2], splat2(-3.0f), D[3]);
            const float2 e0 = __ffma2_rn(__fmul2_rn(t0, k13), t0, __ffma2_rn(t1, t1, eps3));
            const float2 e1 = __ffma2_rn(__fmul2_rn(t2, k13), t2, __ffma2_rn(t3, t3, eps3));
            const float2 e2 = __ffma2_rn(__fmul2_rn(t4, k13), t4, __ffma2_rn(t5, t5, eps3));
            const float mxp = fmaxf(e0.x, fmaxf(e1.x, e2.x)), mnp = fminf(e0.x, fminf(e1.x, e2.x));
            const float mxm = fmaxf(e0.y, fmaxf(e1.y, e2.y)), mnm = fminf(e0.y, fminf(e1.y, e2.y));
            fire[0] = fire[0] || !(mxp > smooth * mnp);
            fire[1] = fire[1] || !(mxm > smooth * mnm);
            nfire += (fire[0] ? 1 : 0) + (fire[1] ? 1 : 0);
        }
        // the network on the rows that use its weights only: the warp's
        // '+' rows, then its '-' rows, packed to the front of the batch (one
        // 16-byte store per row), evaluated in as many 16-row tiles as they
        // fill (rows are independent, so each row's weights are the same)
        const unsigned full = 0xffffffffu, lt = (1u << lane) - 1u;
        const unsigned mp = __ballot_sync(full, !fire[0]), mm = __ballot_sync(full, !fire[1]);
        const int npl = __popc(mp), nrow = npl + __popc(mm);
        float2 w0 = splat2(0.0f), w2 = splat2(0.0f);
        if (nrow > 0) {
            // the network's inputs, normalised, for warps with rows that use it
            float2 mean = V[0];
#pragma unroll
            for (int k = 1; k < 6; k++) mean = __fadd2_rn(mean, V[k]);
            mean = __fmul2_rn(mean, splat2(1.0f / 6.0f));
            float2 dv[6];
            float mxp = 0.f, mxm = 0.f;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                dv[k] = __ffma2_rn(mean, splat2(-1.0f), V[k]);
                mxp = fmaxf(mxp, fabsf(dv[k].x));
                mxm = fmaxf(mxm, fabsf(dv[k].y));
            }
            const float2 inv = make_float2(__fdividef(1.0f, mxp + 1e-12f), __fdividef(1.0f, mxm + 1e-12f));
            float2 x[6];
#pragma unroll
            for (int k = 0; k < 6; k++) x[k] = __fmul2_rn(dv[k], inv);
            const int rp = __popc(mp & lt), rm = npl + __popc(mm & lt);
            if (!fire[0])
                *reinterpret_cast<uint4*>(in + rp * 4) =
                    make_uint4(pack_bf16(x[0].x, x[1].x), pack_bf16(x[2].x, x[3].x), pack_bf16(x[4].x, x[5].x),
                               pack_bf16(1.0f, 0.0f));
            if (!fire[1])
                *reinterpret_cast<uint4*>(in + rm * 4) =
                    make_uint4(pack_bf16(x[0].y, x[1].y), pack_bf16(x[2].y, x[3].y), pack_bf16(x[4].y, x[5].y),
                               pack_bf16(1.0f, 0.0f));
            __syncwarp();
            mlp_warp(W + s * kMlpWords * 32, in, om, lane, (nrow + 15) >> 4);
            __syncwarp();
            if (!fire[0]) { w0.x = om[2 * rp]; w2.x = om[2 * rp + 1]; }
            if (!fire[1]) { w0.y = om[2 * rm]; w2.y = om[2 * rm + 1]; }
            __syncwarp();
        }
        const float2 pp = __ffma2_rn(D[1], splat2(-2.0f), __fadd2_rn(D[0], D[2]));
        const float2 qq = __ffma2_rn(D[2], splat2(-2.0f), __fadd2_rn(D[1], D[3]));
        float2 ph = __ffma2_rn(__fmul2_rn(w0, splat2(1.0f / 3.0f)), pp,
                               __fmul2_rn(__fmul2_rn(__fadd2_rn(w2, splat2(-0.5f)), splat2(1.0f / 6.0f)), qq));
        if (fire[0] || fire[1]) {
            const float2 js = phi_n2(D[0], D[1], D[2], D[3], kEps3);
            if (fire[0]) ph.x = js.x;
            if (fire[1]) ph.y = js.y;
        }
        // phm - php with phm = -(value on -D-)
        return TWICE ? -0.5f * (ph.y + ph.x) : -ph.y - ph.x;
    }
};

template <int AXIS>
__global__ void __launch_bounds__(kLearnedNT, WB_LEARNED_MINB) sweep_learned_kernel(const SweepArgs<float> A,
                                                               const uint32_t* __restrict__ mlp,
                                                               float kappa, float pjump, float smooth) {
    using T = float;
    constexpr int TA = LShape<AXIS>::TA, TP = LShape<AXIS>::TP;
    constexpr int NS = TA + 5;
    constexpr int NC = NS * TP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
#if WB_LEARNED_DELTA
    // weight fragments read from global memory (L1-resident, 32 KB); each
    // thread's back-projection and parked slots after the staged cells
    const uint32_t* Wsm = mlp;
    uint32_t* wbuf = reinterpret_cast<uint32_t*>(sm + (kNSlot * NC + kNThreadSlots * TA * TP));
#else
    uint32_t* Wsm = reinterpret_cast<uint32_t*>(sm + (kNSlot * NC + kNBack * TA * TP));
    uint32_t* wbuf = Wsm + kMlpSmemWords;                 // per warp 256 + 128 words
#endif

    const Tile tile = A.tiles[blockIdx.x];
    const PatchDev P = A.patches[tile.x];
    const int na = AXIS == 0 ? P.nx : (AXIS == 1 ? P.ny : P.nz);
    const int np = AXIS == 0 ? P.ny : P.nx;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;

#if !WB_LEARNED_DELTA
    for (int i = tid; i < kMlpSmemWords; i += TA * TP) Wsm[i] = mlp[i];
#endif

    constexpr int NIT = (NC + TA * TP - 1) / (TA * TP);
    RawCell<T> raw[NIT];
    long long rc[NIT];
    int ridx[NIT];
    bool rok[NIT], rown[NIT];
#pragma unroll
    for (int it = 0; it < NIT; it++) {
        const int e = tid + it * TA * TP;
        int s, tp;
        if (AXIS == 0) { tp = e / NS; s = e - tp * NS; }
        else { s = e / TP; tp = e - s * TP; }
        const int cp = tile.z + tp;
        rok[it] = e < NC && cp < np;
        const int raw_a = tile.y - 3 + s;
        rown[it] = raw_a >= tile.y && raw_a < tile.y + TA && raw_a < na;
        ridx[it] = AXIS == 0 ? tp * NS + s : s * TP + tp;
        if (rok[it]) {
            const int ca = A.links ? raw_a : wrap(raw_a, na);
            int i, j, k;
            if (AXIS == 0) { i = ca; j = cp; k = tile.w; }
            else if (AXIS == 1) { i = cp; j = ca; k = tile.w; }
            else { i = cp; j = tile.w; k = ca; }
            if (A.links) load_cell_linked<T>(A, tile.x, P, i, j, k, raw[it], rc[it]);
            else load_cell<T>(A, P, i, j, k, raw[it], rc[it]);
        }
    }
#pragma unroll
    for (int it = 0; it < NIT; it++)
        if (rok[it]) derive_cell<T, AXIS>(A, raw[it], rc[it], sm, NC, ridx[it], rown[it] && A.er != nullptr);
    __syncthreads();

    const int ta = AXIS == 0 ? threadIdx.x : threadIdx.y;
    const int tp0 = AXIS == 0 ? threadIdx.y : threadIdx.x;
    const int ia = tile.y + ta, ip = tile.z + tp0;
    const bool valid = ia < na && ip < np;
    const int tp = ip < np ? tp0 : 0;                      // stand-in stencil for idle lanes
    int id[6];
#pragma unroll
    for (int m = 0; m < 6; m++) id[m] = (int)chk(AXIS == 0 ? tp * NS + ta + m : (ta + m) * TP + tp, NC, A.flag);
    float pmin = sm[SP_P * NC + id[0]], pmax = pmin;
#pragma unroll
    for (int m = 1; m < 6; m++) {
        const float p = sm[SP_P * NC + id[m]];
        pmin = fminf(pmin, p);
        pmax = fmaxf(pmax, p);
    }
    const int lane = tid & 31, warp = tid >> 5;
    LearnedWeights lw{Wsm, wbuf + warp * 384, reinterpret_cast<float*>(wbuf + warp * 384 + 256), lane,
                      pmax > (1.0f + pjump) * pmin, kappa, smooth};
    T F[7];
    T* bp = sm + kNSlot * NC + tid;
    interface_flux<T, LearnedWeights, WB_LEARNED_DELTA != 0>(sm, NC, id, T(A.gamma), bp, TA * TP, lw, F);
    if (A.lstats) {
        // detector statistics: firings and decisions (7 fields x 2 sides) of
        // the valid interfaces, one pair of atomics per warp
        const unsigned nf = __reduce_add_sync(0xffffffffu, valid ? (unsigned)lw.nfire : 0u);
        const unsigned nv = __reduce_add_sync(0xffffffffu, valid ? 14u : 0u);
        if (lane == 0 && nv) {
            atomicAdd(A.lstats, (unsigned long long)nf);
            atomicAdd(A.lstats + 1, (unsigned long long)nv);
        }
    }
    if (!valid) return;

    int i, j, k;
    if (AXIS == 0) { i = ia; j = ip; k = tile.w; }
    else if (AXIS == 1) { i = ip; j = ia; k = tile.w; }
    else { i = ip; j = tile.w; k = ia; }
    const long long N = A.ncells;
    const long long c = chk(P.off + ((long long)k * P.ny + j) * P.nx + i, N, A.flag);
    T* __restrict__ fo = A.flux;
    T fx, fy, fz;
    if (AXIS == 0) { fx = F[1]; fy = F[2]; fz = F[3]; }
    else if (AXIS == 1) { fy = F[1]; fz = F[2]; fx = F[3]; }
    else { fz = F[1]; fx = F[2]; fy = F[3]; }
    fo[c] = F[0];
    fo[N + c] = fx;
    fo[2 * N + c] = fy;
    fo[3 * N + c] = fz;
    fo[4 * N + c] = F[6];
    fo[5 * N + c] = F[4];
    fo[6 * N + c] = F[5];
}

template <int AXIS>
constexpr size_t learned_smem_bytes() {
    constexpr size_t TA = LShape<AXIS>::TA, TP = LShape<AXIS>::TP;
    constexpr size_t wbuf = sizeof(uint32_t) * (kLearnedNT / 32) * 384;     // per warp 256 + 128 words
#if WB_LEARNED_DELTA
    return sizeof(float) * (kNSlot * (TA + 5) * TP + kNThreadSlots * TA * TP) + wbuf;
#else
    return sizeof(float) * (kNSlot * (TA + 5) * TP + kNBack * TA * TP) + sizeof(uint32_t) * kMlpSmemWords + wbuf;
#endif
}

}  // namespace

void learned_shape(int axis, int* ta, int* tp) {
    *ta = axis == 0 ? LShape<0>::TA : LShape<1>::TA;
    *tp = axis == 0 ? LShape<0>::TP : LShape<1>::TP;
}

cudaError_t prepare_sweep_learned() {
    cudaError_t e;
    e = cudaFuncSetAttribute(sweep_learned_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)learned_smem_bytes<0>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_learned_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)learned_smem_bytes<1>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_learned_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)learned_smem_bytes<2>());
}

cudaError_t launch_sweep_learned(int axis, const SweepArgs<float>& a, int ntiles, const uint32_t* mlp,
                                 float kappa, float pjump, float smooth, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (axis == 0)
        sweep_learned_kernel<0><<<ntiles, dim3(LShape<0>::TA, LShape<0>::TP), learned_smem_bytes<0>(), s>>>(
            a, mlp, kappa, pjump, smooth);
    else if (axis == 1)
        sweep_learned_kernel<1><<<ntiles, dim3(LShape<1>::TP, LShape<1>::TA), learned_smem_bytes<1>(), s>>>(
            a, mlp, kappa, pjump, smooth);
    else
        sweep_learned_kernel<2><<<ntiles, dim3(LShape<2>::TP, LShape<2>::TA), learned_smem_bytes<2>(), s>>>(
            a, mlp, kappa, pjump, smooth);
    return cudaGetLastError();
}

// Host: network parameters (7 x 1379 floats, layout of the public header) to
// the per-lane B-fragment order the kernel reads.
void mlp_fragments(const float* params, uint32_t* out) {
    auto bf = [](float x) -> uint32_t {
        // round to nearest even bfloat16
        uint32_t u;
        memcpy(&u, &x, 4);
        if ((u & 0x7f800000u) == 0x7f800000u) return u >> 16;
        const uint32_t r = 0x7fffu + ((u >> 16) & 1u);
        return (u + r) >> 16;
    };
    auto pk = [&](float lo, float hi) { return bf(lo) | (bf(hi) << 16); };
    auto fbits = [](float x) { uint32_t u; memcpy(&u, &x, 4); return u; };
    const int NH = 32, NIN = 6;
    for (int f = 0; f < WB_MLP_NFIELD; f++) {
        const float* p = params + (size_t)f * WB_MLP_NPARAM;
        const float* W1 = p;
        const float* b1 = W1 + NH * NIN;
        const float* W2 = b1 + NH;
        const float* b2 = W2 + NH * NH;
        const float* W3 = b2 + NH;
        const float* b3 = W3 + 3 * NH;
        // first layer as 32 x 8: six weights, the bias, a zero
        // pre-activations scaled by kGeluK (see gelu_k): first layer (with its
        // bias) and hidden bias times kGeluK, hidden weights halved, output
        // weights divided by 2 kGeluK
        auto w1 = [&](int n, int k) {
            return kGeluK * (k < NIN ? W1[n * NIN + k] : (k == NIN ? b1[n] : 0.f));
        };
        auto w3 = [&](int n, int k) { return n < 3 ? W3[n * NH + k] / (2.0f * kGeluK) : 0.f; };
        for (int lane = 0; lane < 32; lane++) {
            const int g = lane >> 2, t = lane & 3;
            uint32_t* of = out + (size_t)f * kMlpWords * 32;
            auto o = [&](int k) -> uint32_t& { return of[frag_index(k, lane)]; };
            o(34) = 0u;
            o(35) = 0u;
            for (int nt = 0; nt < 4; nt++) o(nt) = pk(w1(8 * nt + g, 2 * t), w1(8 * nt + g, 2 * t + 1));
            for (int nt = 0; nt < 4; nt++)
                for (int kt = 0; kt < 2; kt++) {
                    const int n = 8 * nt + g, k0 = 16 * kt + 2 * t;
                    // hidden weights halved: the layer's input is 2 kGeluK gelu, its
                    // output is wanted times kGeluK
                    o(4 + nt * 4 + kt * 2) = pk(0.5f * W2[n * NH + k0], 0.5f * W2[n * NH + k0 + 1]);
                    o(5 + nt * 4 + kt * 2) = pk(0.5f * W2[n * NH + k0 + 8], 0.5f * W2[n * NH + k0 + 9]);
                }
            for (int kt = 0; kt < 2; kt++) {
                const int k0 = 16 * kt + 2 * t;
                o(20 + kt * 2) = pk(w3(g, k0), w3(g, k0 + 1));
                o(21 + kt * 2) = pk(w3(g, k0 + 8), w3(g, k0 + 9));
            }
            for (int nt = 0; nt < 4; nt++) {
                o(24 + 2 * nt) = fbits(kGeluK * b2[8 * nt + 2 * t]);
                o(25 + 2 * nt) = fbits(kGeluK * b2[8 * nt + 2 * t + 1]);
            }
            o(32) = fbits(2 * t < 3 ? b3[2 * t] : 0.f);
            o(33) = fbits(2 * t + 1 < 3 ? b3[2 * t + 1] : 0.f);
        }
    }
}

size_t mlp_fragment_words() { return (size_t)kMlpSmemWords; }

}  // namespace wb

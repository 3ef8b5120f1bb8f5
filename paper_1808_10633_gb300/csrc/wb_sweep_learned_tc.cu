// wb_sweep_learned_tc.cu -- FP32 WENO5 sweep with learned nonlinear weights,
// the networks evaluated by the 5th-generation tensor cores (tcgen05).
//
// The same scheme as wb_sweep_learned.cu (Sec. 2.1 eq. FWENO with the
// weights (w0, w2) of phi_N from a per-field network 6 -> 32 -> 32 -> 3,
// GELU, softmax, unless a detector fires or the smoothness gate keeps the
// Jiang-Shu weights), with the networks run per block instead of per warp:
//
//  * a block of 128 threads owns 128 interfaces; for each characteristic
//    field the 256 network inputs (two sides per interface) form two
//    M = 128 row tiles, thread t writing row t of both;
//  * one thread issues the three layers as tcgen05.mma (BF16 x BF16 -> FP32,
//    M = 128, N = 32 / 32 / 16, K = 16 / 48 / 32), A from shared memory in
//    the K-major layout without swizzle, B (the weights, all seven fields
//    resident in shared memory) likewise, D in tensor memory; completion is
//    signalled on an mbarrier (tcgen05.commit);
//  * thread t reads its own row back with tcgen05.ld (TMEM lane t), applies
//    the GELU on BF16 pairs and writes the next layer's A row.
// Biases: the first layer's through a constant-1 input column, the hidden
// layer's through two constant-1 columns carrying its BF16 high and low
// parts (together ~16 significant bits), the output layer's added in FP32.
//
// Every mbarrier wait is bounded; a wait that runs out sets kFlagTimeout in
// the grid's status word (reported by the host as WB_ETIMEOUT) and the block
// stops using the tensor cores (Jiang-Shu weights from then on).  TMEM is
// freed before the block exits.
#include "wb_sweep.cuh"

#include <cuda_bf16.h>

namespace wb {
namespace {

constexpr float kGeluKTc = 0.851f;      // gelu(x) = x/2 (1 + tanh(0.851 x)), folded into the weights
constexpr int kTcNT = 128;              // threads = interfaces per block
constexpr int kTcRowsK16 = 128 * 16 * 2;   // bytes of a 128-row tile, K = 16 (BF16)
constexpr int kTcRowsK32 = 128 * 32 * 2;
constexpr int kTcRowsK48 = 128 * 48 * 2;
constexpr int kTcX = 2 * kTcRowsK32;       // two row tiles of layer 3 (layer 1's fit inside)
constexpr int kTcY = 2 * kTcRowsK48;       // two row tiles of layer 2
// per-field weight image (shared memory order): W1 (N 32 x K 16), W2 (N 32 x
// K 48: 32 hidden inputs, the bias high and low parts, zeros), W3 (N 16 x
// K 32, rows 3..15 zero), b3 (4 floats)
constexpr int kTcW1 = 32 * 16 * 2, kTcW2 = 32 * 48 * 2, kTcW3 = 16 * 32 * 2, kTcB3 = 16;
constexpr int kTcField = kTcW1 + kTcW2 + kTcW3 + kTcB3;       // 5136 bytes
constexpr int kTcImage = WB_MLP_NFIELD * kTcField;             // 35952 bytes
constexpr int kTcWait = 1 << 20;        // mbarrier polls before a wait gives up

// Byte offset of element (r, k) of a K-major tile of 16-bit values with K
// columns, no swizzle: 8 x 8 core matrices of 128 contiguous bytes, the
// next 8 columns 128 bytes on (leading byte offset), the next 8 rows
// 16 K bytes on (stride byte offset).
__host__ __device__ constexpr int kmaj(int r, int k, int K) {
    return (r >> 3) * (16 * K) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major tile without swizzle.
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;               // leading byte offset: next 8 columns
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;    // stride byte offset: next 8 rows
    d |= (uint64_t)1 << 46;                         // descriptor version of tcgen05
    return d;                                       // base offset 0, no swizzle
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M.
__device__ __forceinline__ constexpr uint32_t inst_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kTcWait; it++) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 FP32 columns of this thread's TMEM lane.  tcgen05.ld writes its
// registers asynchronously, so the wait is part of the same statement: the
// compiler must not read them, nor give their registers to other values,
// before it has completed.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                 "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                   "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// 4 FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 4; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16_tc(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// 2 k gelu(x) on a BF16 pair from the accumulators y = k x (k folded into
// the stored weights): y + y tanh(y), one tanh and one FMA on the pair.
__device__ __forceinline__ uint32_t gelu_pair(float a, float b) {
    const uint32_t y = pack_bf16_tc(a, b);
    uint32_t t, r;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(y));
    asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(r) : "r"(y), "r"(t));
    return r;
}

// GELU of a 32-wide accumulator row into the row of the next layer's A tile
// (K columns, first 32 of them written).
__device__ __forceinline__ void gelu_row(const float (&v)[32], unsigned char* tile, int row, int K) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
        uint4 q;
        q.x = gelu_pair(v[8 * c + 0], v[8 * c + 1]);
        q.y = gelu_pair(v[8 * c + 2], v[8 * c + 3]);
        q.z = gelu_pair(v[8 * c + 4], v[8 * c + 5]);
        q.w = gelu_pair(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4*>(tile + kmaj(row, 8 * c, K)) = q;
    }
}

// Weight policy of the tensor-core learned scheme (one block, 128 threads,
// every thread calling corr for the same field in the same order).
struct LearnedWeightsTc {
    static constexpr bool kDiff = false;     // works on the stencil values themselves
    const unsigned char* W;   // shared: the seven fields' weight images
    unsigned char* X;         // shared: A of layers 1 and 3 (two row tiles)
    unsigned char* Y;         // shared: A of layer 2 (two row tiles, K = 48)
    volatile int* dead;       // shared: the block gave up on the tensor cores
    unsigned int* flag;       // grid status word
    uint32_t bar;             // mbarrier (shared address)
    uint32_t tmem;            // TMEM base of this block (128 columns)
    int tid;
    bool pfire;               // pressure detector of this interface
    float kappa, smooth;
    uint32_t parity = 0;
    int nfire = 0;            // Jiang-Shu decisions of this thread (fields x sides)

    // thread 0 issues; every thread waits for the layer (bounded).  Returns
    // whether this warp may read the result: the same value on all its lanes
    // (tcgen05.ld is a warp-wide instruction).
    __device__ __forceinline__ bool sync_issue_wait(int s, int layer) {
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (*dead) return false;
        if (tid == 0) {
            fence_after();
            const unsigned char* Wf = W + s * kTcField;
            if (layer == 1) {
                const uint64_t b = mat_desc(smem_addr(Wf), 16 * 16);
#pragma unroll
                for (int q = 0; q < 2; q++)
                    tc_mma(tmem + 32 * q, mat_desc(smem_addr(X + q * kTcRowsK16), 16 * 16), b,
                           inst_desc(128, 32), 0);
            } else if (layer == 2) {
#pragma unroll
                for (int q = 0; q < 2; q++)
#pragma unroll
                    for (int kk = 0; kk < 3; kk++)
                        tc_mma(tmem + 32 * q, mat_desc(smem_addr(Y + q * kTcRowsK48) + 256 * kk, 16 * 48),
                               mat_desc(smem_addr(Wf + kTcW1) + 256 * kk, 16 * 48), inst_desc(128, 32), kk > 0);
            } else {
#pragma unroll
                for (int q = 0; q < 2; q++)
#pragma unroll
                    for (int kk = 0; kk < 2; kk++)
                        tc_mma(tmem + 64 + 16 * q, mat_desc(smem_addr(X + q * kTcRowsK32) + 256 * kk, 16 * 32),
                               mat_desc(smem_addr(Wf + kTcW1 + kTcW2) + 256 * kk, 16 * 32), inst_desc(128, 16),
                               kk > 0);
            }
            tc_commit(bar);
        }
        __syncwarp();            // warp 0 waits once thread 0 has issued
        const bool ok = tc_wait(bar, parity);
        fence_after();
        if (ok) {
            parity ^= 1u;
        } else {                 // parity kept: the final wait is for this phase
            *dead = 1;
            atomicOr(flag, kFlagTimeout);
        }
        return __all_sync(0xffffffffu, ok);
    }

    __device__ __forceinline__ float corr(int s, const float (&w)[6], const float (&g)[6], float alpha) {
        // split fluxes of both sides in packed pairs (lane x '+', lane y '-',
        // its stencil reversed), their differences and the normalised inputs
        const float2 ha = make_float2(0.5f * alpha, -0.5f * alpha);
        float2 V[6];
#pragma unroll
        for (int k = 0; k < 6; k++)
            V[k] = __ffma2_rn(ha, make_float2(w[k], w[5 - k]), __fmul2_rn(splat2(0.5f), make_float2(g[k], g[5 - k])));
        float2 D[4];
#pragma unroll
        for (int k = 0; k < 4; k++) D[k] = __ffma2_rn(V[k], splat2(-1.0f), V[k + 1]);
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
        // layer-1 rows: x0..x5, the bias input 1, zeros
        const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(X + kmaj(tid, 0, 16)) =
            make_uint4(pack_bf16_tc(x[0].x, x[1].x), pack_bf16_tc(x[2].x, x[3].x), pack_bf16_tc(x[4].x, x[5].x),
                       pack_bf16_tc(1.0f, 0.0f));
        *reinterpret_cast<uint4*>(X + kmaj(tid, 8, 16)) = zero;
        *reinterpret_cast<uint4*>(X + kTcRowsK16 + kmaj(tid, 0, 16)) =
            make_uint4(pack_bf16_tc(x[0].y, x[1].y), pack_bf16_tc(x[2].y, x[3].y), pack_bf16_tc(x[4].y, x[5].y),
                       pack_bf16_tc(1.0f, 0.0f));
        *reinterpret_cast<uint4*>(X + kTcRowsK16 + kmaj(tid, 8, 16)) = zero;
        // detectors and the smoothness gate (Jiang-Shu weights where they say so)
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
            const float2 t0 = __ffma2_rn(D[1], splat2(-1.0f), D[0]), t1 = __ffma2_rn(D[1], splat2(-3.0f), D[0]);
            const float2 t2 = __ffma2_rn(D[2], splat2(-1.0f), D[1]), t3 = __fadd2_rn(D[1], D[2]);
            const float2 t4 = __ffma2_rn(D[3], splat2(-1.0f), D[2]),
                         t5 = __ffma2_rn(D[2], splat2(3.0f), __fmul2_rn(D[3], splat2(-1.0f)));
            const float2 is0 = __ffma2_rn(__fmul2_rn(t0, splat2(13.0f)), t0, __fmul2_rn(__fmul2_rn(t1, splat2(3.0f)), t1));
            const float2 is1 = __ffma2_rn(__fmul2_rn(t2, splat2(13.0f)), t2, __fmul2_rn(__fmul2_rn(t3, splat2(3.0f)), t3));
            const float2 is2 = __ffma2_rn(__fmul2_rn(t4, splat2(13.0f)), t4, __fmul2_rn(__fmul2_rn(t5, splat2(3.0f)), t5));
            const float mxp2 = fmaxf(is0.x, fmaxf(is1.x, is2.x)), mnp2 = fminf(is0.x, fminf(is1.x, is2.x));
            const float mxm2 = fmaxf(is0.y, fmaxf(is1.y, is2.y)), mnm2 = fminf(is0.y, fminf(is1.y, is2.y));
            fire[0] = fire[0] || !(mxp2 + 1e-6f > smooth * (mnp2 + 1e-6f));
            fire[1] = fire[1] || !(mxm2 + 1e-6f > smooth * (mnm2 + 1e-6f));
        }
        // the network on the tensor cores, when some thread of the block
        // uses its weights
        const uint32_t lane_base = (uint32_t)(tid & ~31) << 16;      // this warp's TMEM lanes
        float2 w0 = make_float2(0.1f, 0.1f), w2 = make_float2(0.3f, 0.3f);
        fence_async_smem();
        if (__syncthreads_and(fire[0] && fire[1])) {
            nfire += 2;
            const float2 js = phi_n2(D[0], D[1], D[2], D[3]);
            return -js.y - js.x;
        }
        bool live = sync_issue_wait(s, 1);
        if (live) {
#pragma unroll 1
            for (int q = 0; q < 2; q++) {
                float v[32];
                tmem_ld32(tmem + lane_base + 32 * q, v);
                gelu_row(v, Y + q * kTcRowsK48, tid, 48);
            }
        }
        live = sync_issue_wait(s, 2) && live;
        if (live) {
#pragma unroll 1
            for (int q = 0; q < 2; q++) {
                float v[32];
                tmem_ld32(tmem + lane_base + 32 * q, v);
                gelu_row(v, X + q * kTcRowsK32, tid, 32);
            }
        }
        live = sync_issue_wait(s, 3) && live;
        if (live) {
            const float4 b3 = *reinterpret_cast<const float4*>(W + s * kTcField + kTcW1 + kTcW2 + kTcW3);
            float om0[2], om2[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                float z[4];
                tmem_ld4(tmem + lane_base + 64 + 16 * q, z);
                const float z0 = z[0] + b3.x, z1 = z[1] + b3.y, z2 = z[2] + b3.z;
                const float zm = fmaxf(z0, fmaxf(z1, z2));
                const float e0 = __expf(z0 - zm), e1 = __expf(z1 - zm), e2 = __expf(z2 - zm);
                const float r = __fdividef(1.0f, e0 + e1 + e2);
                om0[q] = e0 * r;
                om2[q] = e2 * r;
            }
            w0 = make_float2(om0[0], om0[1]);
            w2 = make_float2(om2[0], om2[1]);
        } else {
            fire[0] = fire[1] = true;
        }
        fence_before();
        nfire += (fire[0] ? 1 : 0) + (fire[1] ? 1 : 0);
        const float2 pp = __ffma2_rn(D[1], splat2(-2.0f), __fadd2_rn(D[0], D[2]));
        const float2 qq = __ffma2_rn(D[2], splat2(-2.0f), __fadd2_rn(D[1], D[3]));
        float2 ph = __ffma2_rn(__fmul2_rn(w0, splat2(1.0f / 3.0f)), pp,
                               __fmul2_rn(__fmul2_rn(__fadd2_rn(w2, splat2(-0.5f)), splat2(1.0f / 6.0f)), qq));
        if (fire[0] || fire[1]) {
            const float2 js = phi_n2(D[0], D[1], D[2], D[3]);
            if (fire[0]) ph.x = js.x;
            if (fire[1]) ph.y = js.y;
        }
        // phm - php with phm = -(value on -D-)
        return -ph.y - ph.x;
    }
};

template <int AXIS>
constexpr int tc_ta() { return shape_ta(AXIS, 0); }

// dynamic shared memory: weight image, X, Y, staged cells, back-projection
// slots, then the mbarrier, TMEM base and the give-up word
template <int AXIS>
constexpr size_t tc_smem_bytes() {
    return (size_t)kTcImage + 16 + kTcX + kTcY +
           sizeof(float) * ((size_t)kNSlot * nc_of(tc_ta<AXIS>()) + (size_t)kNBack * kTcNT) + 32;
}

template <int AXIS>
__global__ void __launch_bounds__(kTcNT, 2) sweep_learned_tc_kernel(const SweepArgs<float> A,
                                                                    const uint4* __restrict__ image,
                                                                    float kappa, float pjump, float smooth) {
    using T = float;
    constexpr int TA = tc_ta<AXIS>(), TP = kTcNT / TA, NS = TA + 5, NC = NS * TP;
    constexpr int LG_TA = TA == 32 ? 5 : (TA == 16 ? 4 : 3);
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* W = tc_smem;
    unsigned char* X = W + kTcImage + 16;                  // 16-byte aligned
    unsigned char* Y = X + kTcX;
    T* sm = reinterpret_cast<T*>(Y + kTcY);
    T* back = sm + kNSlot * NC;
    uint64_t* bar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(back + kNBack * kTcNT) + 7) & ~uintptr_t(7));
    uint32_t* tbase = reinterpret_cast<uint32_t*>(bar + 1);
    int* dead = reinterpret_cast<int*>(tbase + 1);
    const int tid = threadIdx.x, warp = tid >> 5;

    // weights into shared memory; layer-2 A rows: constant columns 32..47
    // (1, 1 for the bias high and low parts, zeros), written once
    for (int i = tid; i < kTcImage / 16; i += kTcNT) reinterpret_cast<uint4*>(W)[i] = image[i];
#pragma unroll
    for (int q = 0; q < 2; q++) {
        *reinterpret_cast<uint4*>(Y + q * kTcRowsK48 + kmaj(tid, 32, 48)) =
            make_uint4(pack_bf16_tc(1.0f, 1.0f), 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(Y + q * kTcRowsK48 + kmaj(tid, 40, 48)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(bar)) : "memory");
        // the initialised barrier visible to the tensor cores' arrivals
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *dead = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" :: "r"(smem_addr(tbase))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }

    // staging (as the Jiang-Shu sweep): cells tile.y-3 .. tile.y+TA+1 of TP pencils
    const Tile tile = A.tiles[blockIdx.x];
    const PatchDev P = A.patches[tile.x & 0xffffff];
    const int na = AXIS == 0 ? P.nx : (AXIS == 1 ? P.ny : P.nz);
    const int np = AXIS == 0 ? P.ny : P.nx;
    constexpr int NIT = (NC + kTcNT - 1) / kTcNT;
    RawCell<T> raw[NIT];
    long long rc[NIT];
    int ridx[NIT];
    bool rok[NIT], rown[NIT];
#pragma unroll
    for (int it = 0; it < NIT; it++) {
        const int e = tid + it * kTcNT;
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
            if (A.links) load_cell_linked<T>(A, tile.x & 0xffffff, P, i, j, k, raw[it], rc[it]);
            else load_cell<T>(A, P, i, j, k, raw[it], rc[it]);
        }
    }
#pragma unroll
    for (int it = 0; it < NIT; it++)
        if (rok[it]) derive_cell<T, AXIS>(A, raw[it], rc[it], sm, NC, ridx[it], rown[it] && A.er != nullptr);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tbase;

    int ta, tp0;
    if (AXIS == 0) { ta = tid & (TA - 1); tp0 = tid >> LG_TA; }
    else { tp0 = tid & (TP - 1); ta = tid >> (7 - LG_TA); }
    const int ia = tile.y + ta, ip = tile.z + tp0;
    const bool valid = ia < na && ip < np;
    const int tp = ip < np ? tp0 : 0;                      // stand-in stencil for idle threads
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
    LearnedWeightsTc lw{W, X, Y, dead, A.flag, smem_addr(bar), tmem, tid, pmax > (1.0f + pjump) * pmin, kappa, smooth};
    T F[7];
    interface_flux<T>(sm, NC, id, T(A.gamma), back + tid, kTcNT, lw, F);
    if (A.lstats) {
        const int lane = tid & 31;
        const unsigned nf = __reduce_add_sync(0xffffffffu, valid ? (unsigned)lw.nfire : 0u);
        const unsigned nv = __reduce_add_sync(0xffffffffu, valid ? 14u : 0u);
        if (lane == 0 && nv) {
            atomicAdd(A.lstats, (unsigned long long)nf);
            atomicAdd(A.lstats + 1, (unsigned long long)nv);
        }
    }
    if (valid) {
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
    // every layer was waited for (or the block gave up: then one more bounded
    // wait for a commit still in flight) before the columns are freed
    fence_before();
    __syncthreads();
    if (*dead && tid == 0) tc_wait(smem_addr(bar), lw.parity);
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" :: "r"(tmem) : "memory");
}

}  // namespace

void learned_tc_shape(int axis, int* ta, int* tp) {
    *ta = shape_ta(axis, 0);
    *tp = kTcNT / *ta;
}

cudaError_t prepare_sweep_learned_tc() {
    cudaError_t e;
    e = cudaFuncSetAttribute(sweep_learned_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_smem_bytes<0>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_learned_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_smem_bytes<1>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_learned_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem_bytes<2>());
}

cudaError_t launch_sweep_learned_tc(int axis, const SweepArgs<float>& a, int ntiles, const void* image,
                                    float kappa, float pjump, float smooth, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    const uint4* img = static_cast<const uint4*>(image);
    if (axis == 0)
        sweep_learned_tc_kernel<0><<<ntiles, kTcNT, tc_smem_bytes<0>(), s>>>(a, img, kappa, pjump, smooth);
    else if (axis == 1)
        sweep_learned_tc_kernel<1><<<ntiles, kTcNT, tc_smem_bytes<1>(), s>>>(a, img, kappa, pjump, smooth);
    else
        sweep_learned_tc_kernel<2><<<ntiles, kTcNT, tc_smem_bytes<2>(), s>>>(a, img, kappa, pjump, smooth);
    return cudaGetLastError();
}

// Host: network parameters (7 x 1379 floats, layout of the public header) to
// the shared-memory image the kernel copies (BF16, K-major tiles), with the
// GELU's constant folded into the weights as in the warp-level kernel.
size_t mlp_tc_image_bytes() { return (size_t)kTcImage; }

void mlp_tc_image(const float* params, unsigned char* out) {
    auto bf = [](float x) -> uint16_t {
        uint32_t u;
        memcpy(&u, &x, 4);
        if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
        return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
    };
    auto unbf = [](uint16_t h) -> float {
        uint32_t u = (uint32_t)h << 16;
        float x;
        memcpy(&x, &u, 4);
        return x;
    };
    const int NH = 32, NIN = 6;
    memset(out, 0, (size_t)kTcImage);
    for (int f = 0; f < WB_MLP_NFIELD; f++) {
        const float* p = params + (size_t)f * WB_MLP_NPARAM;
        const float* W1 = p;
        const float* b1 = W1 + NH * NIN;
        const float* W2 = b1 + NH;
        const float* b2 = W2 + NH * NH;
        const float* W3 = b2 + NH;
        const float* b3 = W3 + 3 * NH;
        unsigned char* o = out + (size_t)f * kTcField;
        auto put = [&](unsigned char* base, int r, int k, int K, float v) {
            const uint16_t h = bf(v);
            memcpy(base + kmaj(r, k, K), &h, 2);
        };
        for (int n = 0; n < NH; n++) {
            for (int k = 0; k < NIN; k++) put(o, n, k, 16, kGeluKTc * W1[n * NIN + k]);
            put(o, n, NIN, 16, kGeluKTc * b1[n]);
            for (int k = 0; k < NH; k++) put(o + kTcW1, n, k, 48, 0.5f * W2[n * NH + k]);
            const float bias = kGeluKTc * b2[n];
            const uint16_t hi = bf(bias);
            put(o + kTcW1, n, 32, 48, unbf(hi));
            put(o + kTcW1, n, 33, 48, bias - unbf(hi));
        }
        for (int n = 0; n < 3; n++)
            for (int k = 0; k < NH; k++) put(o + kTcW1 + kTcW2, n, k, 32, W3[n * NH + k] / (2.0f * kGeluKTc));
        float b[4] = {b3[0], b3[1], b3[2], 0.0f};
        memcpy(o + kTcW1 + kTcW2 + kTcW3, b, sizeof(b));
    }
}

}  // namespace wb

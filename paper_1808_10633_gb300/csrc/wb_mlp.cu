// wb_mlp.cu -- training of the learned WENO weights: one small network per
// characteristic field (6 -> 32 -> 32 -> 3, GELU, softmax) that predicts the
// three nonlinear weights of phi_N (Sec. 2.1) from the normalised stencil.
//
// Records (12 floats): field, x[6] (normalised stencil), q[3] (normalised
// third-order sub-stencil fluxes), T (normalised target reconstruction),
// flag (1 = the jump detector fired; such records are not trained on).
// Loss per record: (sum_k w_k q_k - T)^2 + lam * sum_k d_k log(d_k / w_k).
//
// One training step, all seven networks at once, B records per field:
//   fwd_bwd_kernel   one thread per record: forward pass, loss and the
//                    backward pass to the pre-activation gradients, stored
//                    with the activations in a scratch buffer;
//   reduce_kernel    one thread per parameter (and one per field for the
//                    loss): sums the per-record products in a fixed order, so
//                    the gradient is bitwise repeatable;
//   adam_kernel      one thread per parameter.
// Minibatch indices come from a counter-based generator (splitmix64 of seed,
// step, field, slot), so a run is reproducible.
#include "../../include/wombat_gb300.h"
#include "wb_internal.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace {

constexpr int NIN = 6, NH = 32, NOUT = 3;
constexpr int NP = WB_MLP_NPARAM;            // 1379
constexpr int NF = WB_MLP_NFIELD;            // 7
constexpr int REC = WB_MLP_RECORD;           // 12
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NOUT * NH;
static_assert(O_B3 + NOUT == NP, "parameter layout");

// scratch per record: x(6) a1(32) h1(32) a2(32) h2(32) da1(32) da2(32) dz(3) loss(1)
constexpr int S_X = 0, S_H1 = 6, S_H2 = 38, S_DA1 = 70, S_DA2 = 102, S_DZ = 134, S_L = 137,
              SREC = 138;

// GELU in its sigmoid form, gelu(t) = t sigma(1.702 t) = t/2 (1 + tanh(0.851 t)),
// and its derivative sigma + 1.702 t sigma (1 - sigma).
__device__ __forceinline__ float gelu(float t, float& dgelu) {
    const float sig = 0.5f * (1.0f + tanhf(0.851f * t));
    dgelu = sig + 1.702f * t * sig * (1.0f - sig);
    return t * sig;
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Record index for (field, slot) of this step: either all records of the
// field in order (full batch) or a counter-based random draw.
__device__ __forceinline__ long long pick(const long long* off, const long long* cnt, int f,
                                          int slot, int full, unsigned long long seed,
                                          long long step) {
    if (full) return off[f] + slot;
    const unsigned long long h =
        splitmix64(seed ^ splitmix64((unsigned long long)step * 131071ULL + (unsigned long long)f * 8191ULL +
                                     (unsigned long long)slot));
    return off[f] + (long long)(h % (unsigned long long)cnt[f]);
}

__global__ void __launch_bounds__(128)
fwd_bwd_kernel(const float* __restrict__ rec, const long long* __restrict__ off,
               const long long* __restrict__ cnt, const float* __restrict__ params, int B, int full,
               unsigned long long seed, long long step, float lam, float* __restrict__ scr) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = gid / B, slot = gid - f * B;
    if (f >= NF) return;
    float* s = scr + (long long)gid * SREC;
    if (cnt[f] == 0 || (full && slot >= cnt[f])) {
        for (int t = 0; t < SREC; t++) s[t] = 0.f;
        return;
    }
    const float* r = rec + pick(off, cnt, f, slot, full, seed, step) * REC;
    const float* p = params + (long long)f * NP;
    float x[NIN], a1d[NH], h1[NH], a2d[NH], h2[NH], z[NOUT];
#pragma unroll
    for (int k = 0; k < NIN; k++) x[k] = r[1 + k];
    for (int i = 0; i < NH; i++) {
        float a = p[O_B1 + i];
#pragma unroll
        for (int k = 0; k < NIN; k++) a += p[O_W1 + i * NIN + k] * x[k];
        h1[i] = gelu(a, a1d[i]);
    }
    for (int i = 0; i < NH; i++) {
        float a = p[O_B2 + i];
        for (int k = 0; k < NH; k++) a += p[O_W2 + i * NH + k] * h1[k];
        h2[i] = gelu(a, a2d[i]);
    }
#pragma unroll
    for (int o = 0; o < NOUT; o++) {
        float a = p[O_B3 + o];
        for (int k = 0; k < NH; k++) a += p[O_W3 + o * NH + k] * h2[k];
        z[o] = a;
    }
    const float zm = fmaxf(z[0], fmaxf(z[1], z[2]));
    float e[NOUT], es = 0.f;
#pragma unroll
    for (int o = 0; o < NOUT; o++) { e[o] = expf(z[o] - zm); es += e[o]; }
    float om[NOUT];
#pragma unroll
    for (int o = 0; o < NOUT; o++) om[o] = e[o] / es;
    const float q[NOUT] = {r[7], r[8], r[9]};
    const float T = r[10];
    const float d[NOUT] = {0.1f, 0.6f, 0.3f};
    const float y = om[0] * q[0] + om[1] * q[1] + om[2] * q[2];
    float kl = 0.f;
#pragma unroll
    for (int o = 0; o < NOUT; o++) kl += d[o] * (logf(d[o]) - logf(om[o]));
    const float loss = (y - T) * (y - T) + lam * kl;
    // backward (per record; the mean over records is applied in the reduction)
    float dom[NOUT], sdom = 0.f;
#pragma unroll
    for (int o = 0; o < NOUT; o++) { dom[o] = 2.f * (y - T) * q[o] - lam * d[o] / om[o]; sdom += om[o] * dom[o]; }
    float dz[NOUT];
#pragma unroll
    for (int o = 0; o < NOUT; o++) dz[o] = om[o] * (dom[o] - sdom);
    float da2[NH];
    for (int k = 0; k < NH; k++) {
        float g = 0.f;
#pragma unroll
        for (int o = 0; o < NOUT; o++) g += dz[o] * p[O_W3 + o * NH + k];
        da2[k] = g * a2d[k];
    }
    for (int k = 0; k < NH; k++) {
        float g = 0.f;
        for (int i = 0; i < NH; i++) g += da2[i] * p[O_W2 + i * NH + k];
        s[S_DA1 + k] = g * a1d[k];
    }
#pragma unroll
    for (int k = 0; k < NIN; k++) s[S_X + k] = x[k];
    for (int k = 0; k < NH; k++) {
        s[S_H1 + k] = h1[k];
        s[S_H2 + k] = h2[k];
        s[S_DA2 + k] = da2[k];
    }
#pragma unroll
    for (int o = 0; o < NOUT; o++) s[S_DZ + o] = dz[o];
    s[S_L] = loss;
}

// gradient entry j of field f = (1/n_f) sum over the field's records of the
// product of a pre-activation gradient and an input activation; the loss is
// slot NP of each field.
__global__ void __launch_bounds__(256)
reduce_kernel(const float* __restrict__ scr, const long long* __restrict__ cnt, int B, int full,
              float* __restrict__ grad, float* __restrict__ loss) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = gid / (NP + 1), j = gid - f * (NP + 1);
    if (f >= NF) return;
    const long long nf = full ? (cnt[f] < B ? cnt[f] : B) : (cnt[f] > 0 ? B : 0);
    int ga, gb;     // scratch offsets of the two factors (gb < 0: factor 1)
    if (j < O_B1) { ga = S_DA1 + j / NIN; gb = S_X + j % NIN; }
    else if (j < O_W2) { ga = S_DA1 + (j - O_B1); gb = -1; }
    else if (j < O_B2) { ga = S_DA2 + (j - O_W2) / NH; gb = S_H1 + (j - O_W2) % NH; }
    else if (j < O_W3) { ga = S_DA2 + (j - O_B2); gb = -1; }
    else if (j < O_B3) { ga = S_DZ + (j - O_W3) / NH; gb = S_H2 + (j - O_W3) % NH; }
    else if (j < NP) { ga = S_DZ + (j - O_B3); gb = -1; }
    else { ga = S_L; gb = -1; }
    double acc = 0.0;
    const float* base = scr + (long long)f * B * SREC;
    for (long long r = 0; r < nf; r++) {
        const float* s = base + r * SREC;
        acc += gb < 0 ? double(s[ga]) : double(s[ga]) * double(s[gb]);
    }
    const double v = nf > 0 ? acc / double(nf) : 0.0;
    if (j < NP) grad[(long long)f * NP + j] = float(v);
    else loss[f] = float(v);
}

__global__ void adam_kernel(float* __restrict__ params, const float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

struct Dev {
    float* rec = nullptr;
    long long* off = nullptr;
    long long* cnt = nullptr;
    float* params = nullptr;
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* scr = nullptr;
    float* loss = nullptr;
    ~Dev() {
        for (void* p : {(void*)rec, (void*)off, (void*)cnt, (void*)params, (void*)grad, (void*)m,
                        (void*)v, (void*)scr, (void*)loss})
            if (p) cudaFree(p);
    }
};

// Upload records sorted by field (unflagged only) and the parameters.
int setup(Dev& D, const float* records, long long n, const float* params, int B, int full,
          long long* cnt_out) {
    std::vector<long long> cnt(NF, 0);
    std::vector<std::vector<long long>> by(NF);
    for (long long r = 0; r < n; r++) {
        const int f = (int)records[r * REC];
        if (f < 0 || f >= NF) return wb::set_last_error(WB_EINVAL, "mlp: record with a field outside 0..6");
        if (records[r * REC + 11] != 0.f) continue;
        by[f].push_back(r);
    }
    std::vector<float> sorted;
    std::vector<long long> off(NF, 0);
    long long pos = 0;
    for (int f = 0; f < NF; f++) {
        off[f] = pos;
        cnt[f] = (long long)by[f].size();
        for (long long r : by[f]) sorted.insert(sorted.end(), records + r * REC, records + (r + 1) * REC);
        pos += cnt[f];
    }
    for (int f = 0; f < NF; f++) cnt_out[f] = cnt[f];
    const long long nb = full ? std::max<long long>(1, *std::max_element(cnt.begin(), cnt.end())) : B;
    if (full && nb > (1LL << 24)) return wb::set_last_error(WB_EINVAL, "mlp: too many records per field");
    auto ck = [](cudaError_t e) { return e == cudaSuccess; };
    const size_t rb = sizeof(float) * std::max<size_t>(sorted.size(), REC);
    if (!ck(cudaMalloc(&D.rec, rb)) || !ck(cudaMalloc(&D.off, sizeof(long long) * NF)) ||
        !ck(cudaMalloc(&D.cnt, sizeof(long long) * NF)) ||
        !ck(cudaMalloc(&D.params, sizeof(float) * NF * NP)) ||
        !ck(cudaMalloc(&D.grad, sizeof(float) * NF * NP)) ||
        !ck(cudaMalloc(&D.m, sizeof(float) * NF * NP)) || !ck(cudaMalloc(&D.v, sizeof(float) * NF * NP)) ||
        !ck(cudaMalloc(&D.scr, sizeof(float) * SREC * NF * nb)) ||
        !ck(cudaMalloc(&D.loss, sizeof(float) * NF)))
        return wb::set_last_error(WB_ENOMEM, "mlp: device allocation failed");
    if (!sorted.empty() &&
        !ck(cudaMemcpy(D.rec, sorted.data(), sizeof(float) * sorted.size(), cudaMemcpyHostToDevice)))
        return wb::set_last_error(WB_ECUDA, "mlp: record upload failed");
    if (!ck(cudaMemcpy(D.off, off.data(), sizeof(long long) * NF, cudaMemcpyHostToDevice)) ||
        !ck(cudaMemcpy(D.cnt, cnt.data(), sizeof(long long) * NF, cudaMemcpyHostToDevice)) ||
        !ck(cudaMemcpy(D.params, params, sizeof(float) * NF * NP, cudaMemcpyHostToDevice)) ||
        !ck(cudaMemset(D.m, 0, sizeof(float) * NF * NP)) || !ck(cudaMemset(D.v, 0, sizeof(float) * NF * NP)))
        return wb::set_last_error(WB_ECUDA, "mlp: upload failed");
    return WB_OK;
}

int grad_step(Dev& D, int B, int full, unsigned long long seed, long long step, float lam) {
    const int nrec = NF * B;
    fwd_bwd_kernel<<<(nrec + 127) / 128, 128>>>(D.rec, D.off, D.cnt, D.params, B, full, seed, step, lam, D.scr);
    const int nred = NF * (NP + 1);
    reduce_kernel<<<(nred + 255) / 256, 256>>>(D.scr, D.cnt, B, full, D.grad, D.loss);
    return cudaGetLastError() == cudaSuccess ? WB_OK : wb::set_last_error(WB_ECUDA, "mlp: kernel launch failed");
}

}  // namespace

extern "C" int wb_mlp_loss_grad(const float* records, long long n, const float* params, double lam,
                                double* loss_out, float* grad_out) {
    if (!records || n < 1 || !params || !loss_out || !grad_out)
        return wb::set_last_error(WB_EINVAL, "mlp: null argument or no records");
    Dev D;
    long long cnt[NF];
    int rc = setup(D, records, n, params, 0, 1, cnt);
    if (rc != WB_OK) return rc;
    const long long B = std::max<long long>(1, *std::max_element(cnt, cnt + NF));
    if ((rc = grad_step(D, (int)B, 1, 0, 0, (float)lam)) != WB_OK) return rc;
    float loss[NF];
    if (cudaMemcpy(grad_out, D.grad, sizeof(float) * NF * NP, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(loss, D.loss, sizeof(float) * NF, cudaMemcpyDeviceToHost) != cudaSuccess)
        return wb::set_last_error(WB_ECUDA, "mlp: download failed");
    for (int f = 0; f < NF; f++) loss_out[f] = loss[f];
    return wb::set_last_error(WB_OK, "");
}

extern "C" int wb_mlp_train(const float* records, long long n, float* params, int steps, int batch,
                            double lr, double lam, unsigned long long seed, float* loss_history) {
    if (!records || n < 1 || !params || steps < 0 || batch < 1 || batch > (1 << 20) || !(lr > 0))
        return wb::set_last_error(WB_EINVAL, "mlp: bad training arguments");
    Dev D;
    long long cnt[NF];
    int rc = setup(D, records, n, params, batch, 0, cnt);
    if (rc != WB_OK) return rc;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double p1 = 1.0, p2 = 1.0;
    std::vector<float> hist(NF);
    for (int t = 0; t < steps; t++) {
        if ((rc = grad_step(D, batch, 0, seed, t, (float)lam)) != WB_OK) return rc;
        p1 *= b1;
        p2 *= b2;
        adam_kernel<<<(NF * NP + 255) / 256, 256>>>(D.params, D.grad, D.m, D.v, (float)lr, b1, b2, eps,
                                                    (float)(1.0 - p1), (float)(1.0 - p2), NF * NP);
        if (loss_history) {
            if (cudaMemcpy(hist.data(), D.loss, sizeof(float) * NF, cudaMemcpyDeviceToHost) != cudaSuccess)
                return wb::set_last_error(WB_ECUDA, "mlp: loss download failed");
            for (int f = 0; f < NF; f++) loss_history[(long long)t * NF + f] = hist[f];
        }
    }
    if (cudaMemcpy(params, D.params, sizeof(float) * NF * NP, cudaMemcpyDeviceToHost) != cudaSuccess)
        return wb::set_last_error(WB_ECUDA, "mlp: parameter download failed");
    return wb::set_last_error(WB_OK, "");
}

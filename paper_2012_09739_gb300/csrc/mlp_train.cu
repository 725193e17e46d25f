// Training of the MLP surrogate on (u, |Phi^-1(min(u, 1-u))|) pairs:
// FP16 tensor-core forward and backward (mma.sync m16n8k16, FP32
// accumulation) and Adam on FP32 master weights.
//
// mlp_grad_kernel: each warp takes 64-row chunks of the (mini)batch, runs the
// forward pass of mlp_tc.cuh keeping the activations of each 16-row tile,
// then back-propagates the mean squared error:
//   dy = 2 (y - target) / B
//   dW3 = sum dy h2, db3 = sum dy, dA2 = dy W3 (1 - h2^2), db2 = sum dA2
//   dH1 = dA2 W2 (mma), dA1 = dH1 (1 - h1^2), dW1 = sum dA1 t, db1 = sum dA1
//   dW2 = dA2^T h1 (mma over the rows, operands staged in shared memory and
//         loaded transposed with ldmatrix)
// Per-CTA partial gradients (1153 values + the loss) go to global memory in a
// fixed slot; mlp_adam_kernel sums them in a fixed order (deterministic) and
// applies Adam with bias correction and a cosine learning rate.
#include <math.h>

#include <vector>

#include "api_internal.h"
#include "mlp_tc.cuh"

namespace mlmc {

constexpr int TR_WARPS = 4;
constexpr int PART_STRIDE = 1160;          // 1153 gradients + loss, padded
constexpr int SM_LD = 40;                  // padded row length (halves) of the staging tiles
// Gradient scale: the backward pass works on 2^6 (y - target) (dA2 and the
// tensor-core operands derived from it stay in binary16's normal range even
// for residuals of 1e-5; with the 1 / B factor applied first they were
// binary16 subnormals), and the partials are multiplied by 1 / (2^6 B)
// when written (both factors powers of two for power-of-two batches: exact).
constexpr float GRAD_SCALE = 64.0f;

struct TrainParams {
    float lr0, lr_min, beta1, beta2, eps;
    uint32_t total_steps;
};

__device__ __forceinline__ void ldsm_x4_trans(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                              const __half *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ float quad_sum_rows(float v) {      // sum over lanes with the same L % 4
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

// Rows: full pass (step == nullptr: row r of the batch is pair r) or a
// minibatch of `batch` rows drawn uniformly with replacement with Philox
// (counter (row, step, 0, 'MLP'), key seed).
__global__ void __launch_bounds__(TR_WARPS * 32) mlp_grad_kernel(const MlpWeights *W, const float *u,
                                                                 const float *target, uint64_t n,
                                                                 const uint32_t *step, uint32_t batch, uint32_t k0,
                                                                 uint32_t k1, float inv_batch, float *partials) {
    __shared__ __align__(16) __half sm_h1[TR_WARPS][16 * SM_LD];
    __shared__ __align__(16) __half sm_da[TR_WARPS][16 * SM_LD];
    __shared__ float red[TR_WARPS][PART_STRIDE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;

    MlpFrags F;
    F.load(W);
    const float *W2 = W->w + 64, *W3 = W->w + 64 + 1024 + 32;
    uint32_t w2b[4][2][2];                  // B[k=o][n=j] = W2[o][j]
    float w3c[4][2];                        // W3 of this lane's accumulator columns
    for (int nj = 0; nj < 4; ++nj) {
        const int j = 8 * nj + g;
        for (int kc = 0; kc < 2; ++kc) {
            const int o = 16 * kc + 2 * t;
            w2b[nj][kc][0] = pack_h2(W2[o * 32 + j], W2[(o + 1) * 32 + j]);
            w2b[nj][kc][1] = pack_h2(W2[(o + 8) * 32 + j], W2[(o + 9) * 32 + j]);
        }
        w3c[nj][0] = W3[8 * nj + 2 * t];
        w3c[nj][1] = W3[8 * nj + 2 * t + 1];
    }

    float gw2[2][4][4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c) gw2[a][b][c] = 0.0f;
    float gw1[8] = {}, gb1[8] = {}, gb2[4][2] = {}, gw3[4][2] = {};
    float gb3 = 0.0f, lossp = 0.0f;

    const uint64_t rows = step ? (uint64_t)batch : n;
    const uint32_t s = step ? *step : 0u;
    const uint64_t nchunks = (rows + 63) / 64;
    const uint64_t stride = (uint64_t)gridDim.x * TR_WARPS;
    for (uint64_t ch = (uint64_t)blockIdx.x * TR_WARPS + warp; ch < nchunks; ch += stride) {
        // this lane's two rows: 16 (L % 4) + L / 4 + 8 h
        float tt[2], tg[2], vld[2];
        for (int h = 0; h < 2; ++h) {
            const uint64_t r = ch * 64 + 16 * t + g + 8 * h;
            const bool valid = r < rows;
            uint64_t idx = valid ? r : 0;
            if (step && valid) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)r, s, 0u, 0x4D4C50u), k0, k1);
                idx = n <= 0x100000000ull ? ((uint64_t)w.x * n) >> 32 : (((uint64_t)w.y << 32) | w.x) % n;
            }
            const float ui = u[idx];
            const float v = ui > 0.5f ? __fsub_rn(1.0f, ui) : ui;
            tt[h] = mlp_feature(v);
            tg[h] = target[idx];
            vld[h] = valid ? 1.0f : 0.0f;
        }
#pragma unroll 1
        for (int m = 0; m < 4; ++m) {
            const int src = 4 * g + m;
            const float t0 = __shfl_sync(0xffffffffu, tt[0], src), t1 = __shfl_sync(0xffffffffu, tt[1], src);
            const float tg0 = __shfl_sync(0xffffffffu, tg[0], src), tg1 = __shfl_sync(0xffffffffu, tg[1], src);
            const float v0 = __shfl_sync(0xffffffffu, vld[0], src), v1 = __shfl_sync(0xffffffffu, vld[1], src);
            uint32_t a[2][4], h[2][4];
            mlp_layer1(F, t0, t1, a);
            mlp_layer2(F, a, h);
            float y0, y1;
            mlp_layer3(F, h, y0, y1);
            y0 = __shfl_sync(0xffffffffu, y0, 4 * g);
            y1 = __shfl_sync(0xffffffffu, y1, 4 * g);
            const float r0 = (y0 - tg0) * v0, r1 = (y1 - tg1) * v1;
            if (t == 0) {
                lossp += r0 * r0 + r1 * r1;
                gb3 += GRAD_SCALE * 2.0f * (r0 + r1);
            }
            // scaled residual: keeps dA2 and dH1 in binary16's normal range
            const float dy0 = GRAD_SCALE * 2.0f * r0, dy1 = GRAD_SCALE * 2.0f * r1;
            // layer 3 and tanh of layer 2
            uint32_t da[2][4];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int kc = nt >> 1, hi = nt & 1;
                const float2 h0 = unpack_h2(h[kc][2 * hi]), h1 = unpack_h2(h[kc][2 * hi + 1]);
                gw3[nt][0] += dy0 * h0.x + dy1 * h1.x;
                gw3[nt][1] += dy0 * h0.y + dy1 * h1.y;
                const float a00 = dy0 * w3c[nt][0] * (1.0f - h0.x * h0.x);
                const float a01 = dy0 * w3c[nt][1] * (1.0f - h0.y * h0.y);
                const float a10 = dy1 * w3c[nt][0] * (1.0f - h1.x * h1.x);
                const float a11 = dy1 * w3c[nt][1] * (1.0f - h1.y * h1.y);
                gb2[nt][0] += a00 + a10;
                gb2[nt][1] += a01 + a11;
                da[kc][2 * hi] = pack_h2(a00, a01);
                da[kc][2 * hi + 1] = pack_h2(a10, a11);
            }
            // dH1 = dA2 W2, then layer 1
#pragma unroll
            for (int nj = 0; nj < 4; ++nj) {
                float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, c3 = 0.0f;
                mma16816(c0, c1, c2, c3, da[0][0], da[0][1], da[0][2], da[0][3], w2b[nj][0][0], w2b[nj][0][1], c0,
                         c1, c2, c3);
                mma16816(c0, c1, c2, c3, da[1][0], da[1][1], da[1][2], da[1][3], w2b[nj][1][0], w2b[nj][1][1], c0,
                         c1, c2, c3);
                const int kc = nj >> 1, hi = nj & 1;
                const float2 x0 = unpack_h2(a[kc][2 * hi]), x1 = unpack_h2(a[kc][2 * hi + 1]);
                const float d00 = c0 * (1.0f - x0.x * x0.x), d01 = c1 * (1.0f - x0.y * x0.y);
                const float d10 = c2 * (1.0f - x1.x * x1.x), d11 = c3 * (1.0f - x1.y * x1.y);
                const int i0 = 4 * kc + 2 * hi;
                gw1[i0] += d00 * t0 + d10 * t1;
                gw1[i0 + 1] += d01 * t0 + d11 * t1;
                gb1[i0] += d00 + d10;
                gb1[i0 + 1] += d01 + d11;
            }
            // dW2 = dA2^T h1 over the tile's 16 rows
            __half *sh = sm_h1[warp], *sd = sm_da[warp];
#pragma unroll
            for (int kc = 0; kc < 2; ++kc) {
                const int c = 16 * kc + 2 * t;
                *reinterpret_cast<uint32_t *>(sh + g * SM_LD + c) = a[kc][0];
                *reinterpret_cast<uint32_t *>(sh + (g + 8) * SM_LD + c) = a[kc][1];
                *reinterpret_cast<uint32_t *>(sh + g * SM_LD + c + 8) = a[kc][2];
                *reinterpret_cast<uint32_t *>(sh + (g + 8) * SM_LD + c + 8) = a[kc][3];
                *reinterpret_cast<uint32_t *>(sd + g * SM_LD + c) = da[kc][0];
                *reinterpret_cast<uint32_t *>(sd + (g + 8) * SM_LD + c) = da[kc][1];
                *reinterpret_cast<uint32_t *>(sd + g * SM_LD + c + 8) = da[kc][2];
                *reinterpret_cast<uint32_t *>(sd + (g + 8) * SM_LD + c + 8) = da[kc][3];
            }
            __syncwarp();
            const int mat = lane >> 3, row8 = lane & 7;
#pragma unroll
            for (int mo = 0; mo < 2; ++mo) {
                // A[m=o][k=r] = dA2[r][o]: matrices (rows 0-7 | 8-15) x (cols 16 mo | 16 mo + 8)
                uint32_t a0, a1, a2, a3;
                ldsm_x4_trans(a0, a1, a2, a3, sd + ((mat >> 1) * 8 + row8) * SM_LD + 16 * mo + (mat & 1) * 8);
#pragma unroll
                for (int np = 0; np < 2; ++np) {
                    // B[k=r][n=j] = h1[r][j] for n-tiles 2 np, 2 np + 1
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4_trans(b0, b1, b2, b3, sh + ((mat & 1) * 8 + row8) * SM_LD + 16 * np + (mat >> 1) * 8);
                    float *c = gw2[mo][2 * np];
                    mma16816(c[0], c[1], c[2], c[3], a0, a1, a2, a3, b0, b1, c[0], c[1], c[2], c[3]);
                    float *e = gw2[mo][2 * np + 1];
                    mma16816(e[0], e[1], e[2], e[3], a0, a1, a2, a3, b2, b3, e[0], e[1], e[2], e[3]);
                }
            }
            __syncwarp();
        }
    }

    // ---- warp partials into shared memory in the 1153-value layout
    float *r = red[warp];
    for (int i = lane; i < PART_STRIDE; i += 32) r[i] = 0.0f;
    __syncwarp();
    for (int i = 0; i < 8; ++i) {
        const float sw = quad_sum_rows(gw1[i]), sb = quad_sum_rows(gb1[i]);
        if (g == 0) {
            const int c = MlpFrags::col1(i >> 2, (i >> 1) & 1, i & 1, t);
            r[c] = sw;
            r[32 + c] = sb;
        }
    }
    for (int nt = 0; nt < 4; ++nt)
        for (int e = 0; e < 2; ++e) {
            const float sb2 = quad_sum_rows(gb2[nt][e]), sw3 = quad_sum_rows(gw3[nt][e]);
            if (g == 0) {
                r[64 + 1024 + 8 * nt + 2 * t + e] = sb2;
                r[64 + 1024 + 32 + 8 * nt + 2 * t + e] = sw3;
            }
        }
    for (int mo = 0; mo < 2; ++mo)
        for (int nj = 0; nj < 4; ++nj) {
            const int o0 = 16 * mo + g, j0 = 8 * nj + 2 * t;
            r[64 + o0 * 32 + j0] = gw2[mo][nj][0];
            r[64 + o0 * 32 + j0 + 1] = gw2[mo][nj][1];
            r[64 + (o0 + 8) * 32 + j0] = gw2[mo][nj][2];
            r[64 + (o0 + 8) * 32 + j0 + 1] = gw2[mo][nj][3];
        }
    float b3s = gb3, ls = lossp;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        b3s += __shfl_xor_sync(0xffffffffu, b3s, off);
        ls += __shfl_xor_sync(0xffffffffu, ls, off);
    }
    if (lane == 0) {
        r[1152] = b3s;
        r[1153] = ls;
    }
    __syncthreads();
    const float unscale = inv_batch / GRAD_SCALE;
    for (int i = threadIdx.x; i < PART_STRIDE; i += blockDim.x) {
        float acc = 0.0f;
        for (int w = 0; w < TR_WARPS; ++w) acc += red[w][i];
        partials[(size_t)blockIdx.x * PART_STRIDE + i] = i < MLP_NPARAMS ? acc * unscale : acc;
    }
}

// Sums the CTA partials in a fixed order; then either writes the gradient
// (grad_out != nullptr) or applies one Adam step and advances the step count.
__global__ void __launch_bounds__(1024) mlp_adam_kernel(MlpWeights *W, float *mom, float *vel, const float *partials,
                                                        int nparts, uint32_t *step, TrainParams p, float loss_scale,
                                                        float *loss_out, float *grad_out) {
    const uint32_t s = step ? *step + 1 : 1;   // Adam step, counted from 1
    __syncthreads();
    float lr = p.lr0;
    if (step && p.total_steps > 1) {
        const float frac = fminf((float)(s - 1) / (float)(p.total_steps - 1), 1.0f);
        lr = p.lr_min + 0.5f * (p.lr0 - p.lr_min) * (1.0f + cospif(frac));
    }
    for (int k = threadIdx.x; k < MLP_NPARAMS + 1; k += blockDim.x) {
        float gsum = 0.0f;
        for (int b = 0; b < nparts; ++b) gsum += partials[(size_t)b * PART_STRIDE + k];
        if (k == MLP_NPARAMS) {
            if (loss_out) *loss_out = gsum * loss_scale;
            continue;
        }
        if (grad_out) {
            grad_out[k] = gsum;
            continue;
        }
        const float m = p.beta1 * mom[k] + (1.0f - p.beta1) * gsum;
        const float v = p.beta2 * vel[k] + (1.0f - p.beta2) * gsum * gsum;
        mom[k] = m;
        vel[k] = v;
        const float mhat = m / (1.0f - powf(p.beta1, (float)s));
        const float vhat = v / (1.0f - powf(p.beta2, (float)s));
        W->w[k] -= lr * mhat / (sqrtf(vhat) + p.eps);
    }
    __syncthreads();
    if (step && threadIdx.x == 0) *step = s;
}

// |Phi^-1(min(u, 1-u))| in FP64 for the training targets.
__global__ void mlp_targets_kernel(const float *u, float *z, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double ui = u[i];
        const double v = ui > 0.5 ? 1.0 - ui : ui;
        z[i] = (float)(-normcdfinv(v));
    }
}

cudaError_t mlp_refresh(MlpWeights *m, cudaStream_t s);

namespace {

int grad_grid(const DeviceState &d) {
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, mlp_grad_kernel, TR_WARPS * 32, 0) != cudaSuccess ||
        bps < 1)
        bps = 1;
    return bps * d.sm_count;
}

}  // namespace

}  // namespace mlmc

using namespace mlmc;

extern "C" mlmc_status mlmc_mlp_grad(const float *u_dev, const float *z_dev, size_t n, float *grad_dev,
                                     float *loss_host, void *stream) {
    if (!u_dev || !z_dev || !grad_dev || n == 0) return fail(MLMC_EINVAL, "bad arguments");
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    if (!d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = grad_grid(*d);
    float *partials = nullptr, *loss = nullptr;
    cudaError_t e = cudaMallocAsync(&partials, (size_t)grid * PART_STRIDE * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&loss, sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    mlp_grad_kernel<<<grid, TR_WARPS * 32, 0, s>>>(d->mlp, u_dev, z_dev, n, nullptr, 0, 0, 0, 1.0f / (float)n,
                                                    partials);
    TrainParams p{};
    mlp_adam_kernel<<<1, 1024, 0, s>>>(d->mlp, nullptr, nullptr, partials, grid, nullptr, p, 1.0f / (float)n, loss,
                                       grad_dev);
    e = cudaGetLastError();
    float lh = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lh, loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(partials, s);
    cudaFreeAsync(loss, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mlmc_mlp_grad");
    if (loss_host) *loss_host = lh;
    return MLMC_OK;
}

extern "C" mlmc_status mlmc_mlp_train(const float *u_dev, const float *z_dev, size_t n, const mlmc_train_opts *o,
                                      float *loss_host, void *stream) {
    if (!u_dev || !o || n < 64) return fail(MLMC_EINVAL, "bad arguments (need u_dev, opts, n >= 64)");
    if (o->steps == 0 || o->batch < 64 || o->batch % 64) return fail(MLMC_EINVAL, "steps >= 1, batch a multiple of 64");
    if (!(o->lr0 > 0.0f) || o->lr_min < 0.0f || o->beta1 < 0.0f || o->beta1 >= 1.0f || o->beta2 < 0.0f ||
        o->beta2 >= 1.0f || !(o->eps > 0.0f))
        return fail(MLMC_EINVAL, "invalid optimiser settings");
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    if (!d->mlp_ready) return fail(MLMC_ENOTREADY, "set initial weights with mlmc_mlp_set_weights first");
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = std::min<int>(grad_grid(*d), (int)((o->batch / 64 + TR_WARPS - 1) / TR_WARPS));
    float *partials = nullptr, *mom = nullptr, *vel = nullptr, *loss = nullptr, *targets = nullptr;
    uint32_t *step = nullptr;
    cudaError_t e = cudaMallocAsync(&partials, (size_t)grid * PART_STRIDE * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&mom, 2 * MLP_NPARAMS * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&loss, sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&step, sizeof(uint32_t), s);
    if (e == cudaSuccess && !z_dev) e = cudaMallocAsync(&targets, n * sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    vel = mom + MLP_NPARAMS;
    cudaMemsetAsync(mom, 0, 2 * MLP_NPARAMS * sizeof(float), s);
    cudaMemsetAsync(step, 0, sizeof(uint32_t), s);
    if (!z_dev) {
        mlp_targets_kernel<<<152 * 8, 256, 0, s>>>(u_dev, targets, n);
        z_dev = targets;
    }
    TrainParams p{o->lr0, o->lr_min, o->beta1, o->beta2, o->eps, (uint32_t)std::min<uint64_t>(o->steps, 0xFFFFFFFFu)};
    const uint32_t k0 = (uint32_t)o->seed, k1 = (uint32_t)(o->seed >> 32);
    const float inv_b = 1.0f / (float)o->batch;
    auto enqueue_step = [&](cudaStream_t q) {
        mlp_grad_kernel<<<grid, TR_WARPS * 32, 0, q>>>(d->mlp, u_dev, z_dev, n, step, o->batch, k0, k1, inv_b,
                                                        partials);
        mlp_adam_kernel<<<1, 1024, 0, q>>>(d->mlp, mom, vel, partials, grid, step, p, inv_b, loss, nullptr);
    };
    // the step loop in chunks of 64 steps captured once as a graph
    const uint64_t chunk = 64;
    const uint64_t full = o->steps / chunk, rest = o->steps % chunk;
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    cudaGraphExec_t exec = nullptr;
    if (full > 0) {
        cudaGraph_t graph;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (uint64_t i = 0; i < chunk; ++i) enqueue_step(cs);
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
        }
        for (uint64_t i = 0; i < full && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, s);
    }
    if (e == cudaSuccess) {
        for (uint64_t i = 0; i < rest; ++i) enqueue_step(s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = mlp_refresh(d->mlp, s);
    float lh = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lh, loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(partials, s);
    cudaFreeAsync(mom, s);
    cudaFreeAsync(loss, s);
    cudaFreeAsync(step, s);
    if (targets) cudaFreeAsync(targets, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "mlmc_mlp_train");
    if (loss_host) *loss_host = lh;
    return MLMC_OK;
}

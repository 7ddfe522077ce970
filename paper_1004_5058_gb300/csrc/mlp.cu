// Flow-curve surrogate kernels (include/lbhb_mlp.h): BF16 tensor-core GEMMs
// with FP32 accumulation (mma.sync m16n8k16) and fused epilogues for the
// forward pass, the backward pass and Adam on FP32 master weights.
//
// Every product is written as C[m][n] = sum_k A[m][k] B[n][k] with both operands
// K-contiguous ("NT"): the forward pass multiplies activations [batch][in] by
// weights [out][in]; the backward pass by a transposed weight copy [in][out];
// the weight gradients multiply transposed activation and gradient copies
// [features][batch], which the epilogues write alongside the normal layout.
// Batch rows beyond the live batch are written as zeros, so padded rows and
// columns never contribute.  Weight gradients use split-K partial sums reduced
// in a fixed order, so results are reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbhb_mlp.h"
#include "lb_internal.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int NIN = 5, KIN = 16, HID = 128, NOUT = 2, NOUTP = 16;
constexpr long long OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * NIN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
                    OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID, OFF_W4 = OFF_B3 + HID,
                    OFF_B4 = OFF_W4 + NOUT * HID, NPARAM = OFF_B4 + NOUT;

struct LayerDef {
    int in, in_p, out, out_p;
    long long offW, offB;
};
__host__ __device__ constexpr LayerDef layer_def(int l)
{
    return l == 0   ? LayerDef{NIN, KIN, HID, HID, OFF_W1, OFF_B1}
           : l == 1 ? LayerDef{HID, HID, HID, HID, OFF_W2, OFF_B2}
           : l == 2 ? LayerDef{HID, HID, HID, HID, OFF_W3, OFF_B3}
                    : LayerDef{HID, HID, NOUT, NOUTP, OFF_W4, OFF_B4};
}
constexpr int KSPLIT = 256;  // batch rows per split-K partial of a weight gradient

enum { EPI_TANH = 0, EPI_OUT = 1, EPI_DTANH = 2, EPI_PARTIAL = 3 };

struct Epi {
    const float* bias;  // EPI_TANH, EPI_OUT: [N]
    bf16* out_b;        // EPI_TANH, EPI_DTANH: [rows][ld_out]
    bf16* out_t;        // EPI_TANH, EPI_DTANH: [N][ld_t] (transposed copy)
    float* out_f;       // EPI_OUT: [rows][ld_out]; EPI_PARTIAL: [split][M][N]
    const bf16* hprev;  // EPI_DTANH: activation whose tanh derivative is applied, [rows][ld_out]
    int ld_out, ld_t;
    int rows_live;      // batch rows that hold data; later rows are written as zero
    int rows_buf;       // rows the buffers have
};

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C[m][n] = sum_{k in split} A[m][k] B[n][k]; 64x64 tile per CTA, 4 warps of
// 32x32, BK = 32.  K, the split chunk and both leading dimensions are multiples
// of 8 (16-byte vector loads).
template <int EPI>
__global__ void __launch_bounds__(128) gemm_nt(const bf16* __restrict__ A, int lda, const bf16* __restrict__ B,
                                               int ldb, int M, int N, int K, int kchunk, Epi ep)
{
    __shared__ __align__(16) bf16 As[64][40];
    __shared__ __align__(16) bf16 Bs[64][40];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    for (int k0 = kbeg; k0 < kend; k0 += 32) {
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
            const int c = tid + rep * 128, r = c >> 2, kk = (c & 3) * 8;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (m0 + r < M && k0 + kk < kend) va = *reinterpret_cast<const uint4*>(A + (long long)(m0 + r) * lda + k0 + kk);
            if (n0 + r < N && k0 + kk < kend) vb = *reinterpret_cast<const uint4*>(B + (long long)(n0 + r) * ldb + k0 + kk);
            *reinterpret_cast<uint4*>(&As[r][kk]) = va;
            *reinterpret_cast<uint4*>(&Bs[r][kk]) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < 32; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int rb = wm * 32 + mi * 16;
                a[mi][0] = *reinterpret_cast<const uint32_t*>(&As[rb + g][ks + 2 * t4]);
                a[mi][1] = *reinterpret_cast<const uint32_t*>(&As[rb + g + 8][ks + 2 * t4]);
                a[mi][2] = *reinterpret_cast<const uint32_t*>(&As[rb + g][ks + 2 * t4 + 8]);
                a[mi][3] = *reinterpret_cast<const uint32_t*>(&As[rb + g + 8][ks + 2 * t4 + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int cb = wn * 32 + ni * 8;
                b[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[cb + g][ks + 2 * t4]);
                b[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[cb + g][ks + 2 * t4 + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    mma_bf16(acc[mi][ni], a[mi][0], a[mi][1], a[mi][2], a[mi][3], b[ni][0], b[ni][1]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm * 32 + mi * 16 + g + (r >= 2 ? 8 : 0);
                const int col = n0 + wn * 32 + ni * 8 + 2 * t4 + (r & 1);
                if (col >= N) continue;
                float v = acc[mi][ni][r];
                if (EPI == EPI_PARTIAL) {
                    if (row < M) ep.out_f[((long long)blockIdx.z * M + row) * N + col] = v;
                    continue;
                }
                if (row >= ep.rows_buf) continue;
                const bool live = row < ep.rows_live;
                if (EPI == EPI_TANH) {
                    v = live ? tanhf(v + ep.bias[col]) : 0.f;
                } else if (EPI == EPI_OUT) {
                    v = live ? v + ep.bias[col] : 0.f;
                } else {  // EPI_DTANH
                    const float h = __bfloat162float(ep.hprev[(long long)row * ep.ld_out + col]);
                    v = live ? v * (1.f - h * h) : 0.f;
                }
                if (EPI == EPI_OUT) {
                    ep.out_f[(long long)row * ep.ld_out + col] = v;
                } else {
                    const bf16 hv = __float2bfloat16_rn(v);
                    ep.out_b[(long long)row * ep.ld_out + col] = hv;
                    ep.out_t[(long long)col * ep.ld_t + row] = hv;
                }
            }
}

// z = (x - center) / half_range, padded to 16 columns, both layouts.
__global__ void normalise_kernel(const float* __restrict__ x, int B, int Bbuf, const float* __restrict__ center,
                                 const float* __restrict__ half, bf16* __restrict__ z, bf16* __restrict__ zt)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bbuf) return;
    for (int c = 0; c < KIN; ++c) {
        float v = 0.f;
        if (b < B && c < NIN) v = (x[b * NIN + c] - center[c]) / half[c];
        const bf16 hv = __float2bfloat16_rn(v);
        z[(long long)b * KIN + c] = hv;
        zt[(long long)c * Bbuf + b] = hv;
    }
}

__device__ __forceinline__ float bce_logits(float z, float y)
{
    return fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
}

// dL/dy for y = (stress/scale, logit); per-block loss partials (FP64).
__global__ void loss_grad_kernel(const float* __restrict__ out, const float* __restrict__ target,
                                 const float* __restrict__ label, int B, int Bbuf, float inv_scale, float lam,
                                 bf16* __restrict__ d, bf16* __restrict__ dt, double* __restrict__ part)
{
    __shared__ double red[256];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < Bbuf) {
        float d0 = 0.f, d1 = 0.f;
        if (b < B) {
            const float y0 = out[(long long)b * NOUTP + 0], y1 = out[(long long)b * NOUTP + 1];
            const float t = target[b] * inv_scale, lab = label[b];
            const float e = y0 - t;
            l = (double)(e * e) + (double)lam * (double)bce_logits(y1, lab);
            d0 = 2.f * e / (float)B;
            const float sg = 1.f / (1.f + expf(-y1));
            d1 = lam * (sg - lab) / (float)B;
        }
        for (int c = 0; c < NOUTP; ++c) {
            const float v = c == 0 ? d0 : (c == 1 ? d1 : 0.f);
            const bf16 hv = __float2bfloat16_rn(v);
            d[(long long)b * NOUTP + c] = hv;
            dt[(long long)c * Bbuf + b] = hv;
        }
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void loss_finish_kernel(const double* __restrict__ part, int n, int B, float* __restrict__ loss_f,
                                   double* __restrict__ loss_d)
{
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    s /= (double)B;
    if (loss_f) *loss_f = (float)s;
    if (loss_d) *loss_d = s;
}

// grad[offW + o*in + i] = sum_s part[s][o][i] for the live block (o < out, i < in).
__global__ void reduce_wgrad_kernel(const float* __restrict__ part, int S, int Mo, int Ni, int out, int in,
                                    float* __restrict__ grad)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= out * in) return;
    const int o = k / in, i = k % in;
    float s = 0.f;
    for (int p = 0; p < S; ++p) s += part[((long long)p * Mo + o) * Ni + i];
    grad[k] = s;
}

// grad_b[o] = sum over live batch rows of d[o][b] (transposed gradient rows): a
// block of BIAS_THREADS per output o, each thread a strided part of the batch,
// then a fixed-shape tree (the same order every call).
constexpr int BIAS_THREADS = 256;
__global__ void __launch_bounds__(BIAS_THREADS) bias_grad_kernel(const bf16* __restrict__ dt, int Bbuf, int B,
                                                                 float* __restrict__ grad)
{
    const int o = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < B; b += BIAS_THREADS) s += __bfloat162float(dt[(long long)o * Bbuf + b]);
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) s += __shfl_down_sync(0xffffffffu, s, w);
    __shared__ float warp_sum[BIAS_THREADS / 32];
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < BIAS_THREADS / 32; ++k) t += warp_sum[k];
        grad[o] = t;
    }
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);
}

// FP32 masters -> padded BF16 weights [out_p][in_p], their transposes, padded FP32 biases.
__global__ void refresh_kernel(const float* __restrict__ p, bf16* w1, bf16* w1t, bf16* w2, bf16* w2t, bf16* w3,
                               bf16* w3t, bf16* w4, bf16* w4t, float* b1, float* b2, float* b3, float* b4)
{
    bf16* W[4] = {w1, w2, w3, w4};
    bf16* Wt[4] = {w1t, w2t, w3t, w4t};
    float* Bp[4] = {b1, b2, b3, b4};
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int base = 0;
    for (int l = 0; l < 4; ++l) {
        const LayerDef L = layer_def(l);
        const int nw = L.out_p * L.in_p;
        if (k >= base && k < base + nw) {
            const int o = (k - base) / L.in_p, i = (k - base) % L.in_p;
            const float v = (o < L.out && i < L.in) ? p[L.offW + (long long)o * L.in + i] : 0.f;
            const bf16 hv = __float2bfloat16_rn(v);
            W[l][o * L.in_p + i] = hv;
            Wt[l][i * L.out_p + o] = hv;
        }
        base += nw;
        if (k >= base && k < base + L.out_p) {
            const int o = k - base;
            Bp[l][o] = o < L.out ? p[L.offB + o] : 0.f;
        }
        base += L.out_p;
    }
}

__global__ void output_kernel(const float* __restrict__ out, int B, float scale, float* __restrict__ y)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    y[2 * b] = out[(long long)b * NOUTP] * scale;
    y[2 * b + 1] = out[(long long)b * NOUTP + 1];
}

constexpr int MAX_BINS = 256;  // bins of the serving error-budget table

}  // namespace

// ------------------------------------------------------------- serving --
// The whole serving call in one kernel: a CTA takes 64 queries through the
// normalisation, the three tanh layers and the output layer with every
// activation kept in shared memory (each warp owns 16 rows), the layer's
// weights staged in shared memory, then makes the fallback decision.  The
// products are the GEMM kernel's, tile for tile: one m16n8k16 BF16 product per
// 16-wide slice of K in increasing K, bias and tanh in FP32, activations
// rounded to BF16; so the served values equal the layered forward pass bit for
// bit.
constexpr int SRV_ROWS = 64, SRV_LD = HID + 8;  // padded rows: no bank conflicts on fragment loads
// two activation buffers and two weight buffers (the next layer's weights are
// copied while the current layer computes)
constexpr size_t SRV_SMEM = sizeof(bf16) * (2 * SRV_ROWS * SRV_LD + 2 * HID * SRV_LD);

// 16-byte asynchronous global -> shared copies, in commit groups
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Weights of layer l into a padded shared buffer, by all 128 threads.
__device__ __forceinline__ void stage_weights(bf16* Ws, const bf16* W, int l, int tid)
{
    const LayerDef L = layer_def(l);
    for (int e = tid; e < L.out_p * (L.in_p / 8); e += 128) {
        const int n = e / (L.in_p / 8), k8 = (e % (L.in_p / 8)) * 8;
        cp_async16(&Ws[n * SRV_LD + k8], W + (long long)n * L.in_p + k8);
    }
}

struct ServeArgs {
    const float* x;
    int B;
    const bf16* W[4];
    const float* bias[4];
    const float *center, *half;
    float scale, margin;
    const int* over_budget;
    int n_bins;
    float ls_lo, ls_hi;
    float *stress, *logit;
    int* fallback;
};

__global__ void __launch_bounds__(128) serve_fused_kernel(ServeArgs a)
{
    extern __shared__ __align__(16) unsigned char srv_smem[];
    bf16* act0 = reinterpret_cast<bf16*>(srv_smem);
    bf16* act1 = act0 + SRV_ROWS * SRV_LD;
    bf16* const wbuf0 = act1 + SRV_ROWS * SRV_LD;
    bf16* const wbuf1 = wbuf0 + HID * SRV_LD;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int b0 = blockIdx.x * SRV_ROWS, r0 = warp * 16;
    // the first two layers' weights start copying at once
    stage_weights(wbuf0, a.W[0], 0, tid);
    cp_async_commit();
    stage_weights(wbuf1, a.W[1], 1, tid);
    cp_async_commit();

    // z = (x - center) / half_range, padded to KIN columns (zero rows past B)
    for (int e = tid; e < SRV_ROWS * KIN; e += 128) {
        const int r = e / KIN, c = e % KIN, b = b0 + r;
        float v = 0.f;
        if (b < a.B && c < NIN) v = (a.x[b * NIN + c] - a.center[c]) / a.half[c];
        act0[r * SRV_LD + c] = __float2bfloat16_rn(v);
    }
    bf16* in = act0;
    bf16* out = act1;
    for (int l = 0; l < 4; ++l) {
        const LayerDef L = layer_def(l);
        const bf16* Ws = (l & 1) ? wbuf1 : wbuf0;
        if (l < 3)
            cp_async_wait<1>();  // this layer's group is done, the next one may still fly
        else
            cp_async_wait<0>();
        __syncthreads();  // weights and input activations visible to all warps
        constexpr int NT = HID / 8;
        float acc[NT][4];
#pragma unroll
        for (int ni = 0; ni < NT; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[ni][r] = 0.f;
        const int nt = L.out_p / 8;
        for (int ks = 0; ks < L.in_p; ks += 16) {
            const uint32_t x0 = *reinterpret_cast<const uint32_t*>(&in[(r0 + g) * SRV_LD + ks + 2 * t4]);
            const uint32_t x1 = *reinterpret_cast<const uint32_t*>(&in[(r0 + g + 8) * SRV_LD + ks + 2 * t4]);
            const uint32_t x2 = *reinterpret_cast<const uint32_t*>(&in[(r0 + g) * SRV_LD + ks + 2 * t4 + 8]);
            const uint32_t x3 = *reinterpret_cast<const uint32_t*>(&in[(r0 + g + 8) * SRV_LD + ks + 2 * t4 + 8]);
#pragma unroll
            for (int ni = 0; ni < NT; ++ni) {
                if (ni >= nt) break;
                const uint32_t w0 = *reinterpret_cast<const uint32_t*>(&Ws[(ni * 8 + g) * SRV_LD + ks + 2 * t4]);
                const uint32_t w1 = *reinterpret_cast<const uint32_t*>(&Ws[(ni * 8 + g) * SRV_LD + ks + 2 * t4 + 8]);
                mma_bf16(acc[ni], x0, x1, x2, x3, w0, w1);
            }
        }
        if (l < 3) {
#pragma unroll
            for (int ni = 0; ni < NT; ++ni)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int row = r0 + g + (r >= 2 ? 8 : 0), col = ni * 8 + 2 * t4 + (r & 1);
                    out[row * SRV_LD + col] = __float2bfloat16_rn(tanhf(acc[ni][r] + a.bias[l][col]));
                }
            __syncwarp();  // a warp reads back only its own rows
            bf16* t = in;
            in = out;
            out = t;
            if (l + 2 < 4) {
                __syncthreads();  // every warp is done with this layer's weights
                stage_weights((l & 1) ? wbuf1 : wbuf0, a.W[l + 2], l + 2, tid);
                cp_async_commit();
            }
        } else {
            // columns 0 (stress / scale) and 1 (logit) sit in n-tile 0: lanes with t4 == 0
            if (t4 == 0) {
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int row = r0 + g + 8 * h2, b = b0 + row;
                    if (b >= a.B) continue;
                    const float y0 = acc[0][2 * h2] + a.bias[3][0], y1 = acc[0][2 * h2 + 1] + a.bias[3][1];
                    bool outside = false;
                    for (int c = 0; c < NIN; ++c) {
                        const float xv = a.x[b * NIN + c];
                        outside |= !(fabsf(xv - a.center[c]) <= a.half[c]);
                    }
                    bool budget = false;
                    if (a.n_bins > 0) {
                        const float ls = a.x[b * NIN];
                        int k = (int)floorf((ls - a.ls_lo) / (a.ls_hi - a.ls_lo) * a.n_bins);
                        k = k < 0 ? 0 : (k >= a.n_bins ? a.n_bins - 1 : k);
                        budget = a.over_budget[k] != 0;
                    }
                    a.stress[b] = y0 * a.scale;
                    a.logit[b] = y1;
                    a.fallback[b] = (outside || budget || !(fabsf(y1) >= a.margin)) ? 1 : 0;
                }
            }
        }
    }
}

struct mlp_handle {
    mlp_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int bbuf = 0;  // batch rows of the buffers (max_batch rounded up to 64)
    int splits = 0;
    float *P = nullptr, *M = nullptr, *V = nullptr, *G = nullptr;
    bf16 *W[4] = {}, *Wt[4] = {};
    float* bias[4] = {};
    bf16 *Z = nullptr, *Zt = nullptr;
    bf16 *H[3] = {}, *Ht[3] = {};
    float* OUT = nullptr;
    bf16 *D[4] = {}, *Dt[4] = {};  // gradients w.r.t. pre-activations of layers 1..3, and the output
    float* part = nullptr;         // split-K partials
    double* loss_part = nullptr;
    double* loss_d = nullptr;
    float *center = nullptr, *half = nullptr;
    int* over_budget = nullptr;  // [MAX_BINS]
    int n_bins = 0;
    float ls_lo = 0.f, ls_hi = 1.f;
    long long adam_t = 0;
    long long launches = 0;
    std::vector<void*> allocs;
};

namespace {

void release(mlp_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs) cudaFree(p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

template <class T>
cudaError_t alloc(mlp_handle* h, T** p, size_t n)
{
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e == cudaSuccess) {
        h->allocs.push_back(*p);
        e = cudaMemsetAsync(*p, 0, n * sizeof(T), h->stream);
    }
    return e;
}

int rows8(int B) { return (B + 7) / 8 * 8; }

template <int EPI>
cudaError_t gemm(mlp_handle* h, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, int kchunk,
                 const Epi& ep)
{
    const int splits = (K + kchunk - 1) / kchunk;
    dim3 grid((M + 63) / 64, (N + 63) / 64, splits);
    gemm_nt<EPI><<<grid, 128, 0, h->stream>>>(A, lda, B, ldb, M, N, K, kchunk, ep);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t forward(mlp_handle* h, const float* x, int B)
{
    const int Br = rows8(B), bb = h->bbuf;
    normalise_kernel<<<(bb + 127) / 128, 128, 0, h->stream>>>(x, B, bb, h->center, h->half, h->Z, h->Zt);
    h->launches++;
    const bf16* in = h->Z;
    int ld_in = KIN;
    for (int l = 0; l < 4; ++l) {
        const LayerDef L = layer_def(l);
        Epi ep{};
        ep.bias = h->bias[l];
        ep.rows_live = B;
        ep.rows_buf = bb;
        cudaError_t e;
        if (l < 3) {
            ep.out_b = h->H[l];
            ep.out_t = h->Ht[l];
            ep.ld_out = HID;
            ep.ld_t = bb;
            e = gemm<EPI_TANH>(h, in, ld_in, h->W[l], L.in_p, Br, L.out_p, L.in_p, L.in_p, ep);
            in = h->H[l];
            ld_in = HID;
        } else {
            ep.out_f = h->OUT;
            ep.ld_out = NOUTP;
            e = gemm<EPI_OUT>(h, in, ld_in, h->W[l], L.in_p, Br, L.out_p, L.in_p, L.in_p, ep);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Loss gradient and backpropagation into h->G (flat FP32 gradient).
cudaError_t backward(mlp_handle* h, const float* target, const float* label, int B, float* loss_f, double* loss_d)
{
    const int Br = rows8(B), bb = h->bbuf;
    const int nblk = (bb + 255) / 256;
    loss_grad_kernel<<<nblk, 256, 0, h->stream>>>(h->OUT, target, label, B, bb, (float)(1.0 / h->cfg.sigma_scale),
                                                   (float)h->cfg.lam, h->D[3], h->Dt[3], h->loss_part);
    loss_finish_kernel<<<1, 32, 0, h->stream>>>(h->loss_part, nblk, B, loss_f, loss_d);
    h->launches += 2;
    for (int l = 3; l >= 0; --l) {
        const LayerDef L = layer_def(l);
        const bf16* xt = l == 0 ? h->Zt : h->Ht[l - 1];  // layer input, transposed [in_p][bb]
        // weight gradient: dW[o][i] = sum_b D_l[b][o] X[b][i]
        Epi ep{};
        ep.out_f = h->part;
        cudaError_t e = gemm<EPI_PARTIAL>(h, h->Dt[l], bb, xt, bb, L.out_p, L.in_p, Br, KSPLIT, ep);
        if (e != cudaSuccess) return e;
        const int S = (Br + KSPLIT - 1) / KSPLIT;
        reduce_wgrad_kernel<<<(L.out * L.in + 255) / 256, 256, 0, h->stream>>>(h->part, S, L.out_p, L.in_p, L.out,
                                                                                L.in, h->G + L.offW);
        bias_grad_kernel<<<L.out, BIAS_THREADS, 0, h->stream>>>(h->Dt[l], bb, B, h->G + L.offB);
        h->launches += 2;
        if (l > 0) {
            // D_{l-1} = (D_l W_l) * (1 - h_{l-1}^2)
            Epi ed{};
            ed.out_b = h->D[l - 1];
            ed.out_t = h->Dt[l - 1];
            ed.hprev = h->H[l - 1];
            ed.ld_out = HID;
            ed.ld_t = bb;
            ed.rows_live = B;
            ed.rows_buf = bb;
            e = gemm<EPI_DTANH>(h, h->D[l], L.out_p, h->Wt[l], L.out_p, Br, L.in_p, L.out_p, L.out_p, ed);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

cudaError_t refresh(mlp_handle* h)
{
    int total = 0;
    for (int l = 0; l < 4; ++l) total += layer_def(l).out_p * layer_def(l).in_p + layer_def(l).out_p;
    refresh_kernel<<<(total + 255) / 256, 256, 0, h->stream>>>(h->P, h->W[0], h->Wt[0], h->W[1], h->Wt[1], h->W[2],
                                                                h->Wt[2], h->W[3], h->Wt[3], h->bias[0], h->bias[1],
                                                                h->bias[2], h->bias[3]);
    h->launches++;
    return cudaGetLastError();
}

lb_status invalid(const char* msg)
{
    lbhb::set_handleless_error(msg);
    return LB_ERR_INVALID;
}

lb_status check_batch(const mlp_handle* h, int B)
{
    if (B >= 1 && B <= h->cfg.max_batch) return LB_OK;
    char buf[128];
    snprintf(buf, sizeof buf, "mlp: batch %d outside 1..max_batch (%d)", B, h->cfg.max_batch);
    lbhb::set_handleless_error(buf);
    return LB_ERR_INVALID;
}

}  // namespace

extern "C" {

long long mlp_param_count(void) { return NPARAM; }

lb_status mlp_create(const mlp_config* cfg, void* cuda_stream, mlp_handle** out)
{
    if (!out || !cfg) return invalid("mlp_create: NULL config or output");
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_batch > (1 << 24) || !(cfg->sigma_scale > 0.0) || !(cfg->lr >= 0.0))
        return invalid("mlp_create: max_batch, sigma_scale or lr out of range");
    for (int c = 0; c < NIN; ++c)
        if (!(cfg->half_range[c] > 0.0) || !std::isfinite(cfg->center[c]))
            return invalid("mlp_create: half_range must be > 0 and center finite");
    mlp_handle* h = new (std::nothrow) mlp_handle();
    if (!h) return LB_ERR_NOMEM;
    h->cfg = *cfg;
    cudaGetDevice(&h->device);
    cudaError_t e = cudaSuccess;
    if (cuda_stream) h->stream = (cudaStream_t)cuda_stream;
    else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        h->own_stream = e == cudaSuccess;
    }
    h->bbuf = (cfg->max_batch + 63) / 64 * 64;
    const int bb = h->bbuf;
    h->splits = (bb + KSPLIT - 1) / KSPLIT;
    if (e == cudaSuccess) e = alloc(h, &h->P, NPARAM);
    if (e == cudaSuccess) e = alloc(h, &h->M, NPARAM);
    if (e == cudaSuccess) e = alloc(h, &h->V, NPARAM);
    if (e == cudaSuccess) e = alloc(h, &h->G, NPARAM);
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        e = alloc(h, &h->W[l], (size_t)layer_def(l).out_p * layer_def(l).in_p);
        if (e == cudaSuccess) e = alloc(h, &h->Wt[l], (size_t)layer_def(l).out_p * layer_def(l).in_p);
        if (e == cudaSuccess) e = alloc(h, &h->bias[l], (size_t)layer_def(l).out_p);
    }
    if (e == cudaSuccess) e = alloc(h, &h->Z, (size_t)bb * KIN);
    if (e == cudaSuccess) e = alloc(h, &h->Zt, (size_t)bb * KIN);
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
        e = alloc(h, &h->H[l], (size_t)bb * HID);
        if (e == cudaSuccess) e = alloc(h, &h->Ht[l], (size_t)bb * HID);
        if (e == cudaSuccess) e = alloc(h, &h->D[l], (size_t)bb * HID);
        if (e == cudaSuccess) e = alloc(h, &h->Dt[l], (size_t)bb * HID);
    }
    if (e == cudaSuccess) e = alloc(h, &h->D[3], (size_t)bb * NOUTP);
    if (e == cudaSuccess) e = alloc(h, &h->Dt[3], (size_t)bb * NOUTP);
    if (e == cudaSuccess) e = alloc(h, &h->OUT, (size_t)bb * NOUTP);
    if (e == cudaSuccess) e = alloc(h, &h->part, (size_t)h->splits * HID * HID);
    if (e == cudaSuccess) e = alloc(h, &h->loss_part, (size_t)(bb + 255) / 256);
    if (e == cudaSuccess) e = alloc(h, &h->loss_d, 1);
    if (e == cudaSuccess) e = alloc(h, &h->center, NIN);
    if (e == cudaSuccess) e = alloc(h, &h->half, NIN);
    if (e == cudaSuccess)  // the fused serving kernel keeps activations and weights in shared memory
        e = cudaFuncSetAttribute(serve_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SRV_SMEM);
    if (e == cudaSuccess) e = alloc(h, &h->over_budget, MAX_BINS);
    if (e == cudaSuccess) {
        float c[NIN], hr[NIN];
        for (int i = 0; i < NIN; ++i) {
            c[i] = (float)cfg->center[i];
            hr[i] = (float)cfg->half_range[i];
        }
        e = cudaMemcpyAsync(h->center, c, sizeof c, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->half, hr, sizeof hr, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(h);
        return e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA;
    }
    *out = h;
    return LB_OK;
}

lb_status mlp_set_params(mlp_handle* h, const float* params, long long n)
{
    if (!h || !params || n != NPARAM) return invalid("mlp: NULL handle or parameters, or wrong count");
    cudaError_t e = cudaMemcpyAsync(h->P, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->M, 0, sizeof(float) * NPARAM, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->V, 0, sizeof(float) * NPARAM, h->stream);
    if (e == cudaSuccess) e = refresh(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->adam_t = 0;
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_get_params(mlp_handle* h, float* params, long long n)
{
    if (!h || !params || n != NPARAM) return invalid("mlp: NULL handle or parameters, or wrong count");
    cudaError_t e = cudaMemcpyAsync(params, h->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_forward(mlp_handle* h, const float* x, int batch, float* out)
{
    if (!h || !x || !out) return invalid("mlp: NULL handle or buffer");
    if (check_batch(h, batch) != LB_OK) return LB_ERR_INVALID;
    cudaError_t e = forward(h, x, batch);
    if (e == cudaSuccess) {
        output_kernel<<<(batch + 255) / 256, 256, 0, h->stream>>>(h->OUT, batch, (float)h->cfg.sigma_scale, out);
        h->launches++;
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_gradients(mlp_handle* h, const float* x, const float* target_stress, const float* label, int batch,
                        float* grad, double* loss)
{
    if (!h || !x || !target_stress || !label || !grad) return invalid("mlp: NULL handle or buffer");
    if (check_batch(h, batch) != LB_OK) return LB_ERR_INVALID;
    cudaError_t e = forward(h, x, batch);
    if (e == cudaSuccess) e = backward(h, target_stress, label, batch, nullptr, h->loss_d);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, h->G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, h->stream);
    double l = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, h->loss_d, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (loss) *loss = l;
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_train_step(mlp_handle* h, const float* x, const float* target_stress, const float* label, int batch,
                         float* loss_dev)
{
    if (!h || !x || !target_stress || !label) return invalid("mlp: NULL handle or buffer");
    if (check_batch(h, batch) != LB_OK) return LB_ERR_INVALID;
    cudaError_t e = forward(h, x, batch);
    if (e == cudaSuccess) e = backward(h, target_stress, label, batch, loss_dev, nullptr);
    if (e == cudaSuccess) {
        h->adam_t++;
        const double b1 = h->cfg.beta1, b2 = h->cfg.beta2;
        const float c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)h->adam_t)));
        const float c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)h->adam_t)));
        adam_kernel<<<(int)((NPARAM + 255) / 256), 256, 0, h->stream>>>(h->P, h->M, h->V, h->G, NPARAM,
                                                                        (float)h->cfg.lr, (float)b1, (float)b2,
                                                                        (float)h->cfg.eps, c1, c2);
        h->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = refresh(h);
    return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_serve(mlp_handle* h, const float* x, int batch, float* stress, float* logit, int* fallback)
{
    if (!h || !x || !stress || !logit || !fallback) return invalid("mlp: NULL handle or buffer");
    if (check_batch(h, batch) != LB_OK) return LB_ERR_INVALID;
    ServeArgs a{};
    a.x = x;
    a.B = batch;
    for (int l = 0; l < 4; ++l) {
        a.W[l] = h->W[l];
        a.bias[l] = h->bias[l];
    }
    a.center = h->center;
    a.half = h->half;
    a.scale = (float)h->cfg.sigma_scale;
    a.margin = (float)h->cfg.logit_margin;
    a.over_budget = h->over_budget;
    a.n_bins = h->n_bins;
    a.ls_lo = h->ls_lo;
    a.ls_hi = h->ls_hi;
    a.stress = stress;
    a.logit = logit;
    a.fallback = fallback;
    serve_fused_kernel<<<(batch + SRV_ROWS - 1) / SRV_ROWS, 128, SRV_SMEM, h->stream>>>(a);
    h->launches++;
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

lb_status mlp_set_error_budget(mlp_handle* h, const float* bin_error, int n_bins, double log_s_lo,
                               double log_s_hi, double budget)
{
    if (!h || n_bins < 0 || n_bins > MAX_BINS || (n_bins > 0 && (!bin_error || !(log_s_hi > log_s_lo))))
        return invalid("mlp_set_error_budget: NULL handle, n_bins outside 0..256 or empty log S range");
    int flags[MAX_BINS] = {0};
    for (int k = 0; k < n_bins; ++k) flags[k] = !(bin_error[k] <= budget);  // NaN error is over budget
    cudaError_t e = cudaMemcpyAsync(h->over_budget, flags, sizeof(int) * MAX_BINS, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return LB_ERR_CUDA;
    h->n_bins = n_bins;
    h->ls_lo = (float)log_s_lo;
    h->ls_hi = (float)log_s_hi;
    return LB_OK;
}

long long mlp_kernel_launches(const mlp_handle* h) { return h ? h->launches : 0; }

void mlp_destroy(mlp_handle* h) { release(h); }

}  // extern "C"

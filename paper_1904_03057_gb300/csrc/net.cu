// net.cu -- the learned preconditioner of flexible CG: a small 3-level 3-D convolutional network,
// its BF16 forward / backward kernels (FP32 accumulation), Adam, and the C ABI (bsk_net_*).
//
// The network maps a normalised residual r (fine grid, 1 channel) to an error estimate z:
//   a1 = relu(down(r; W1) + b1)                 1 -> 16 channels, stride-2 3^3 conv   (L1)
//   a2 = relu(conv_s2(a1; W2) + b2)             16 -> 16, stride 2                    (L2)
//   a3 = relu(conv_s1(a2; W3) + b3)             16 -> 16, stride 1                    (L2)
//   a4 = relu(convT_s2(a3; W4) + b4 + a1)       16 -> 16, transposed stride 2 + skip  (L1)
//   z  = mask * (up(a4; W5) + b5 + conv_s1(r; Wf))  16 -> 1 transposed stride 2, plus a
//                                               full-resolution 3^3 filter of r      (L0)
// With BSK_ACT_LINEAR relu is the identity and the biases are dropped: the network is then a
// linear multilevel map of r (the form that works as a flexible-CG preconditioner).
// Activations are BF16, channels-last (16 channels = 32 bytes per voxel). The 16 -> 16
// convolutions run on the tensor cores (mma.sync m16n8k16 BF16 -> FP32, implicit GEMM over the
// 27 taps); the 1-channel ends and the weight gradients run on the FP32 pipes. The paper has no
// learned component: this is the workload's addition to the CG stage of section 2.5.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include <cuda_bf16.h>

#include "bsk.h"
#include "bsk_launch.h"

namespace {

enum ConvMode : int { CONV_S1 = 0, CONV_S2 = 1, CONVT_S2 = 2 };

constexpr int C = 16;       // channels of the hidden layers
constexpr int KT = 27;      // 3^3 taps

// parameter block layout (FP32 master copy), offsets in floats
constexpr int OFF_W1 = 0;                       // [27][16]        (tap, co)
constexpr int OFF_B1 = OFF_W1 + KT * C;
constexpr int OFF_W2 = OFF_B1 + C;              // [27][16][16]    (tap, co, ci)
constexpr int OFF_B2 = OFF_W2 + KT * C * C;
constexpr int OFF_W3 = OFF_B2 + C;
constexpr int OFF_B3 = OFF_W3 + KT * C * C;
constexpr int OFF_W4 = OFF_B3 + C;
constexpr int OFF_B4 = OFF_W4 + KT * C * C;
constexpr int OFF_W5 = OFF_B4 + C;              // [27][16]        (tap, ci)
constexpr int OFF_B5 = OFF_W5 + KT * C;
constexpr int OFF_WF = OFF_B5 + 1;              // [27]            full-resolution 1 -> 1 filter
constexpr int NPARAM = OFF_WF + KT;

// Source index along one axis of output index o through tap k (0..2); -1 if none.
__device__ __forceinline__ int src_index(int mode, int o, int k, int nin)
{
    int i;
    if (mode == CONV_S1) i = o + k - 1;
    else if (mode == CONV_S2) i = 2 * o + k - 1;
    else {
        const int t = o + 1 - k;
        if (t & 1) return -1;
        i = t >> 1;
    }
    return (i >= 0 && i < nin) ? i : -1;
}

struct D3 { int nx, ny, nz; };

// ---- 16 -> 16 convolution on the tensor cores -------------------------------------------------
// out[o][co] = act( sum_{taps k, ci} W[k][co][ci] in[src(o,k)][ci] + bias[co] + skip[o][co] )
// One warp computes 16 output voxels (consecutive x, or x of one parity for the transposed
// convolution) x 16 channels with two m16n8k16 MMAs per tap.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int MODE>
__global__ void __launch_bounds__(128) k_conv16(const __nv_bfloat16* __restrict__ in, D3 din,
                                                __nv_bfloat16* __restrict__ out, D3 dout,
                                                const __nv_bfloat16* __restrict__ W,
                                                const float* __restrict__ bias,
                                                const __nv_bfloat16* __restrict__ skip, int relu)
{
    __shared__ uint32_t sW[KT * C * C / 2];   // [tap][co][ci pairs]
    const uint32_t* Wg = reinterpret_cast<const uint32_t*>(W);
    for (int i = threadIdx.x; i < KT * C * C / 2; i += blockDim.x) sW[i] = Wg[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    // tiles: per output row (z, y): for the transposed conv two parity classes of x
    const int xstep = MODE == CONVT_S2 ? 2 : 1;
    const int per_class = MODE == CONVT_S2 ? (dout.nx + 1) / 2 : dout.nx;
    const int tiles_class = (per_class + 15) / 16;
    const int tiles_row = tiles_class * xstep;
    const long long ntiles = (long long)tiles_row * dout.ny * dout.nz;
    const long long tile = (long long)blockIdx.x * 4 + warp;
    if (tile >= ntiles) return;
    const int tr = (int)(tile % tiles_row);
    const long long row = tile / tiles_row;
    const int oy = (int)(row % dout.ny), oz = (int)(row / dout.ny);
    const int parity = MODE == CONVT_S2 ? tr / tiles_class : 0;
    const int ox0 = (tr % tiles_class) * 16 * xstep + parity;
    const int oxa = ox0 + xstep * g, oxb = ox0 + xstep * (g + 8);   // this lane's two rows

    const uint32_t* inw = reinterpret_cast<const uint32_t*>(in);
    float acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    for (int kz = 0; kz < 3; kz++) {
        const int iz = src_index(MODE, oz, kz, din.nz);
        if (iz < 0) continue;
        for (int ky = 0; ky < 3; ky++) {
            const int iy = src_index(MODE, oy, ky, din.ny);
            if (iy < 0) continue;
            const long long rowbase = ((long long)iz * din.ny + iy) * din.nx;
#pragma unroll
            for (int kx = 0; kx < 3; kx++) {
                const int ixa = oxa < dout.nx ? src_index(MODE, oxa, kx, din.nx) : -1;
                const int ixb = oxb < dout.nx ? src_index(MODE, oxb, kx, din.nx) : -1;
                if (__all_sync(0xffffffffu, ixa < 0 && ixb < 0)) continue;
                uint32_t a[4];
                const long long va = (rowbase + ixa) * (C / 2), vb = (rowbase + ixb) * (C / 2);
                a[0] = ixa >= 0 ? __ldg(inw + va + t) : 0u;
                a[1] = ixb >= 0 ? __ldg(inw + vb + t) : 0u;
                a[2] = ixa >= 0 ? __ldg(inw + va + t + 4) : 0u;
                a[3] = ixb >= 0 ? __ldg(inw + vb + t + 4) : 0u;
                const int k = (kz * 3 + ky) * 3 + kx;
#pragma unroll
                for (int nb = 0; nb < 2; nb++) {
                    const uint32_t* wb = sW + (k * C + nb * 8 + g) * (C / 2);
                    mma_bf16(acc[nb], a, wb[t], wb[t + 4]);
                }
            }
        }
    }
    // epilogue: rows g and g+8, channels nb*8 + 2t, +1
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int ox = h ? oxb : oxa;
        if (ox >= dout.nx) continue;
        const long long o = ((long long)oz * dout.ny + oy) * dout.nx + ox;
#pragma unroll
        for (int nb = 0; nb < 2; nb++) {
            const int co = nb * 8 + 2 * t;
            float v0 = acc[nb][2 * h], v1 = acc[nb][2 * h + 1];
            if (bias) { v0 += bias[co]; v1 += bias[co + 1]; }
            if (skip) {
                const __nv_bfloat162 s = reinterpret_cast<const __nv_bfloat162*>(skip + o * C)[co / 2];
                v0 += __bfloat162float(s.x);
                v1 += __bfloat162float(s.y);
            }
            if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
            reinterpret_cast<__nv_bfloat162*>(out + o * C)[co / 2] = __floats2bfloat162_rn(v0, v1);
        }
    }
}

// ---- 1-channel ends (FP32 pipes) ----------------------------------------------------------
// out[o][c] = act( sum_k W[k][c] x[2o + k - 1] + bias[c] ), x fine (FP32, 1 channel), out coarse.
__global__ void k_down1(const float* __restrict__ x, D3 din, __nv_bfloat16* __restrict__ out, D3 dout,
                        const float* __restrict__ W, const float* __restrict__ bias, int relu)
{
    __shared__ float sW[KT * C];
    for (int i = threadIdx.x; i < KT * C; i += blockDim.x) sW[i] = W[i];
    __syncthreads();
    const long long n = (long long)dout.nx * dout.ny * dout.nz;
    const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int ox = (int)(o % dout.nx), oy = (int)((o / dout.nx) % dout.ny), oz = (int)(o / ((long long)dout.nx * dout.ny));
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; c++) acc[c] = bias ? bias[c] : 0.f;
    for (int kz = 0; kz < 3; kz++) {
        const int iz = src_index(CONV_S2, oz, kz, din.nz);
        if (iz < 0) continue;
        for (int ky = 0; ky < 3; ky++) {
            const int iy = src_index(CONV_S2, oy, ky, din.ny);
            if (iy < 0) continue;
            for (int kx = 0; kx < 3; kx++) {
                const int ix = src_index(CONV_S2, ox, kx, din.nx);
                if (ix < 0) continue;
                const float v = x[((long long)iz * din.ny + iy) * din.nx + ix];
                const float* w = sW + ((kz * 3 + ky) * 3 + kx) * C;
#pragma unroll
                for (int c = 0; c < C; c++) acc[c] = fmaf(w[c], v, acc[c]);
            }
        }
    }
    __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(out + o * C);
#pragma unroll
    for (int c = 0; c < C; c += 2) {
        float v0 = acc[c], v1 = acc[c + 1];
        if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
        dst[c / 2] = __floats2bfloat162_rn(v0, v1);
    }
}

// Output layer, z[o] = mask * ( sum_{k valid} sum_c W[k][c] a[srcT(o,k)][c] + b
//                                 + sum_k Wf[k] r[o + k - 1] ), a coarse (BF16), z and r fine.
// One thread per 2 x 2 x 2 block of fine voxels (2m .. 2m+1 per axis), which gathers from the
// 2 x 2 x 2 coarse voxels m .. m+1, so that each coarse voxel is loaded once for the eight
// outputs it feeds. Along an axis, fine 2m + e
// takes coarse m + d with tap k = e + 1 - 2d (the transposed stride-2 gather of src_index:
// (e, d) = (0, 0) -> 1, (1, 0) -> 2, (1, 1) -> 0, (0, 1) none).
__global__ void __launch_bounds__(128) k_up1b(const __nv_bfloat16* __restrict__ a, D3 din, float* __restrict__ z,
                                              D3 dout, const float* __restrict__ W,
                                              const float* __restrict__ bias, const uint8_t* __restrict__ mask,
                                              const float* __restrict__ r, const float* __restrict__ Wf)
{
    __shared__ float sW[KT * C];
    __shared__ float sF[KT];
    for (int i = threadIdx.x; i < KT * C; i += blockDim.x) sW[i] = W[i];
    for (int i = threadIdx.x; i < KT; i += blockDim.x) sF[i] = Wf[i];
    __syncthreads();
    const long long nb = (long long)din.nx * din.ny * din.nz;
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int mx = (int)(b % din.nx), my = (int)((b / din.nx) % din.ny), mz = (int)(b / ((long long)din.nx * din.ny));
    int act = 0;   // bit e: fine output e = (ez, ey, ex) exists and is active
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int fz = 2 * mz + (e >> 2), fy = 2 * my + ((e >> 1) & 1), fx = 2 * mx + (e & 1);
        if (fz < dout.nz && fy < dout.ny && fx < dout.nx) {
            const long long o = ((long long)fz * dout.ny + fy) * dout.nx + fx;
            if (!mask || mask[o]) act |= 1 << e;
            else z[o] = 0.f;
        }
    }
    if (!act) return;
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; e++) acc[e] = 0.f;
#pragma unroll
    for (int d = 0; d < 8; d++) {
        const int dz = d >> 2, dy = (d >> 1) & 1, dx = d & 1;
        const int cz = mz + dz, cy = my + dy, cx = mx + dx;
        if (cz >= din.nz || cy >= din.ny || cx >= din.nx) continue;
        const uint4* av = reinterpret_cast<const uint4*>(a + (((long long)cz * din.ny + cy) * din.nx + cx) * C);
        const uint4 v0 = av[0], v1 = av[1];   // 16 BF16 channels
        const uint32_t wv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        float f[C];
#pragma unroll
        for (int c = 0; c < C / 2; c++) {
            const float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wv[c]));
            f[2 * c] = t.x;
            f[2 * c + 1] = t.y;
        }
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int ez = e >> 2, ey = (e >> 1) & 1, ex = e & 1;
            if ((dz && !ez) || (dy && !ey) || (dx && !ex)) continue;   // no tap joins them
            if (!(act & (1 << e))) continue;
            const int kz = ez + 1 - 2 * dz, ky = ey + 1 - 2 * dy, kx = ex + 1 - 2 * dx;
            const float* w = sW + ((kz * 3 + ky) * 3 + kx) * C;
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int c = 0; c < C; c += 2) {
                s0 = fmaf(w[c], f[c], s0);
                s1 = fmaf(w[c + 1], f[c + 1], s1);
            }
            acc[e] += s0 + s1;
        }
    }
    const float b5 = bias ? bias[0] : 0.f;
#pragma unroll
    for (int e = 0; e < 8; e++) {
        if (!(act & (1 << e))) continue;
        const int fz = 2 * mz + (e >> 2), fy = 2 * my + ((e >> 1) & 1), fx = 2 * mx + (e & 1);
        float fine = 0.f;   // the full-resolution filter of r
        for (int kz = 0; kz < 3; kz++) {
            const int iz = fz + kz - 1;
            if (iz < 0 || iz >= dout.nz) continue;
            for (int ky = 0; ky < 3; ky++) {
                const int iy = fy + ky - 1;
                if (iy < 0 || iy >= dout.ny) continue;
                const float* rr = r + ((long long)iz * dout.ny + iy) * dout.nx;
#pragma unroll
                for (int kx = 0; kx < 3; kx++) {
                    const int ix = fx + kx - 1;
                    if (ix >= 0 && ix < dout.nx) fine = fmaf(sF[(kz * 3 + ky) * 3 + kx], rr[ix], fine);
                }
            }
        }
        z[((long long)fz * dout.ny + fy) * dout.nx + fx] = acc[e] + b5 + fine;
    }
}

// dWf[k] += sum_o dz[o] r[o + k - 1] (fine grid, FP32)
__global__ void k_wgrad_fine(const float* __restrict__ dz, const float* __restrict__ r, D3 d,
                             float* __restrict__ dWf)
{
    __shared__ float s[KT][128];
    float acc[KT];
#pragma unroll
    for (int k = 0; k < KT; k++) acc[k] = 0.f;
    const long long n = (long long)d.nx * d.ny * d.nz;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const float g = dz[o];
        if (g == 0.f) continue;
        const int ox = (int)(o % d.nx), oy = (int)((o / d.nx) % d.ny), oz = (int)(o / ((long long)d.nx * d.ny));
        for (int k = 0; k < KT; k++) {
            const int iz = src_index(CONV_S1, oz, k / 9, d.nz), iy = src_index(CONV_S1, oy, (k / 3) % 3, d.ny),
                      ix = src_index(CONV_S1, ox, k % 3, d.nx);
            if (iz >= 0 && iy >= 0 && ix >= 0) acc[k] = fmaf(g, r[((long long)iz * d.ny + iy) * d.nx + ix], acc[k]);
        }
    }
    for (int k = 0; k < KT; k++) s[k][threadIdx.x] = acc[k];
    __syncthreads();
    if (threadIdx.x < KT) {
        float t = 0.f;
        for (int i = 0; i < 128; i++) t += s[threadIdx.x][i];
        atomicAdd(&dWf[threadIdx.x], t);
    }
}

// ---- weight gradients (FP32 pipes, FP32 accumulation, atomics into dW) ---------------------
// dW[k][co][ci] += sum_o g[o][co] in[src(o,k)][ci]; thread = (co, ci), 27 taps each.
template <int MODE>
__global__ void __launch_bounds__(256) k_wgrad16(const __nv_bfloat16* __restrict__ in, D3 din,
                                                 const __nv_bfloat16* __restrict__ g, D3 dout,
                                                 float* __restrict__ dW, int chunk)
{
    __shared__ float sg[8][C];
    __shared__ float sin_[8][KT][C];
    const int co = threadIdx.x >> 4, ci = threadIdx.x & 15;
    float acc[KT];
#pragma unroll
    for (int k = 0; k < KT; k++) acc[k] = 0.f;
    const long long n = (long long)dout.nx * dout.ny * dout.nz;
    const long long o0 = (long long)blockIdx.x * chunk;
    const long long o1 = o0 + chunk < n ? o0 + chunk : n;
    for (long long ob = o0; ob < o1; ob += 8) {
        __syncthreads();
        // stage 8 output voxels: their gradients and the 27 source voxels of each
        for (int i = threadIdx.x; i < 8 * C; i += 256) {
            const long long o = ob + i / C;
            sg[i / C][i % C] = o < o1 ? __bfloat162float(g[o * C + i % C]) : 0.f;
        }
        for (int i = threadIdx.x; i < 8 * KT * C; i += 256) {
            const int vv = i / (KT * C), k = (i / C) % KT, c = i % C;
            const long long o = ob + vv;
            float val = 0.f;
            if (o < o1) {
                const int ox = (int)(o % dout.nx), oy = (int)((o / dout.nx) % dout.ny),
                          oz = (int)(o / ((long long)dout.nx * dout.ny));
                const int iz = src_index(MODE, oz, k / 9, din.nz), iy = src_index(MODE, oy, (k / 3) % 3, din.ny),
                          ix = src_index(MODE, ox, k % 3, din.nx);
                if (iz >= 0 && iy >= 0 && ix >= 0)
                    val = __bfloat162float(in[(((long long)iz * din.ny + iy) * din.nx + ix) * C + c]);
            }
            sin_[vv][k][c] = val;
        }
        __syncthreads();
#pragma unroll
        for (int vv = 0; vv < 8; vv++) {
            const float gv = sg[vv][co];
#pragma unroll
            for (int k = 0; k < KT; k++) acc[k] = fmaf(gv, sin_[vv][k][ci], acc[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < KT; k++)
        if (acc[k] != 0.f) atomicAdd(&dW[(k * C + co) * C + ci], acc[k]);
}

// dW[k][c] += sum_o G[o][c] X[2o + k - 1]: G coarse 16-channel (BF16), X fine 1-channel (FP32).
// (dW1 with G = layer-1 gradient, X = r; dW5 with G = a4, X = dz.)
__global__ void k_wgrad1(const __nv_bfloat16* __restrict__ G, D3 dc, const float* __restrict__ X, D3 df,
                         float* __restrict__ dW, int chunk)
{
    const int t = threadIdx.x;   // 432 active: (k, c)
    const int k = t / C, c = t % C;
    if (t >= KT * C) return;
    const long long n = (long long)dc.nx * dc.ny * dc.nz;
    const long long o0 = (long long)blockIdx.x * chunk;
    const long long o1 = o0 + chunk < n ? o0 + chunk : n;
    float acc = 0.f;
    for (long long o = o0; o < o1; o++) {
        const int ox = (int)(o % dc.nx), oy = (int)((o / dc.nx) % dc.ny), oz = (int)(o / ((long long)dc.nx * dc.ny));
        const int iz = src_index(CONV_S2, oz, k / 9, df.nz), iy = src_index(CONV_S2, oy, (k / 3) % 3, df.ny),
                  ix = src_index(CONV_S2, ox, k % 3, df.nx);
        if (iz < 0 || iy < 0 || ix < 0) continue;
        acc = fmaf(__bfloat162float(G[o * C + c]), X[((long long)iz * df.ny + iy) * df.nx + ix], acc);
    }
    if (acc != 0.f) atomicAdd(&dW[k * C + c], acc);
}

// ---- elementwise helpers -------------------------------------------------------------------
// g *= (a > 0) (relu != 0; identity otherwise), both 16-channel BF16; optionally also adds g
// into acc (the skip connection).
__global__ void k_relu_bwd(__nv_bfloat16* __restrict__ g, const __nv_bfloat16* __restrict__ a, long long n,
                           __nv_bfloat16* __restrict__ skip_acc, int relu)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v = (!relu || __bfloat162float(a[i]) > 0.f) ? __bfloat162float(g[i]) : 0.f;
        g[i] = __float2bfloat16(v);
        if (skip_acc) skip_acc[i] = __float2bfloat16(__bfloat162float(skip_acc[i]) + v);
    }
}

// db[c] += sum over voxels of g[o][c] (16 channels, BF16) -- or of a 1-channel FP32 field.
__global__ void k_bias_grad16(const __nv_bfloat16* __restrict__ g, long long nvox, float* __restrict__ db)
{
    __shared__ float s[256];
    const int c = threadIdx.x & 15;
    float acc = 0.f;
    for (long long v = blockIdx.x * 16LL + (threadIdx.x >> 4); v < nvox; v += gridDim.x * 16LL)
        acc += __bfloat162float(g[v * C + c]);
    s[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < 16) {
        float tot = 0.f;
        for (int i = threadIdx.x; i < 256; i += 16) tot += s[i];
        atomicAdd(&db[c], tot);
    }
}

// dz = w (z - e) mask, w = 2 / count; loss += w/2 * sum (z - e)^2 over active voxels; db5 += sum dz.
__global__ void k_loss(const float* __restrict__ z, const float* __restrict__ e, const uint8_t* __restrict__ mask,
                       long long n, float w, float* __restrict__ dz, float* __restrict__ loss, float* __restrict__ db5)
{
    __shared__ float s1[256], s2[256];
    float l = 0.f, b = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float act = (!mask || mask[i]) ? 1.f : 0.f;
        const float d = (z[i] - e[i]) * act;
        dz[i] = w * d;
        l += d * d;
        b += w * d;
    }
    s1[threadIdx.x] = l;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) { s1[threadIdx.x] += s1[threadIdx.x + st]; s2[threadIdx.x] += s2[threadIdx.x + st]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(loss, 0.5f * w * s1[0]);
        if (db5) atomicAdd(db5, s2[0]);
    }
}

// dz = w * g on active voxels (an output gradient supplied by the caller), db5 += sum dz.
__global__ void k_given_grad(const float* __restrict__ g, const uint8_t* __restrict__ mask, long long n, float w,
                             float* __restrict__ dz, float* __restrict__ db5)
{
    __shared__ float s2[256];
    float b = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = (!mask || mask[i]) ? w * g[i] : 0.f;
        dz[i] = d;
        b += d;
    }
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) s2[threadIdx.x] += s2[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0 && db5) atomicAdd(db5, s2[0]);
}

// Adam on the FP32 master parameters; grads are summed over the mini-batch (scale = 1/batch).
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, int n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2, float scale)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gr = grad[i] * scale;
    const float mi = b1 * m[i] + (1.f - b1) * gr;
    const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// BF16 weight copies for the forward pass and for the input gradients:
//   fwd[k][co][ci] = W[k][co][ci]; trn[k][ci][co] = W[k][co][ci] (transposed);
//   flip[k][ci][co] = W[26 - k][co][ci] (transposed and tap-flipped, stride-1 adjoint).
__global__ void k_prep_weights(const float* __restrict__ W, __nv_bfloat16* __restrict__ fwd,
                               __nv_bfloat16* __restrict__ trn, __nv_bfloat16* __restrict__ flip)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= KT * C * C) return;
    const int k = i / (C * C), co = (i / C) % C, ci = i % C;
    const __nv_bfloat16 w = __float2bfloat16(W[i]);
    fwd[i] = w;
    if (trn) trn[(k * C + ci) * C + co] = w;
    if (flip) flip[((KT - 1 - k) * C + ci) * C + co] = w;
}

// master weights of the 1-channel ends, rounded to BF16 values (kept as FP32 for the FP32 pipes)
__global__ void k_round_bf16(const float* __restrict__ src, float* __restrict__ dst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __bfloat162float(__float2bfloat16(src[i]));
}

int blocks_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

// ---- the network object ----------------------------------------------------------------------
struct bsk_net {
    D3 d0, d1, d2;
    cudaStream_t stream;
    float *params, *grad, *adam_m, *adam_v;      // FP32, NPARAM each
    float* w_round;                              // BF16-rounded copies of W1, W5 (FP32 storage)
    __nv_bfloat16 *w2, *w3, *w4, *w2t, *w3f, *w4t;   // BF16 weights of the tensor-core layers
    __nv_bfloat16 *a1, *a2, *a3, *a4;            // activations
    __nv_bfloat16 *g1, *g2, *g3, *g4;            // activation gradients
    float *z, *dz, *loss;                        // output, output gradient, loss accumulator
    int adam_t;
    int linear;                                  // BSK_ACT_LINEAR: identity activations, no biases
};

namespace {

int nfail(int code, const char* msg) { return bsk::set_error(code, msg); }

#define NCUDA(call)                                                        \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return nfail(BSK_ECUDA, #call " failed");   \
    } while (0)

D3 halfdims(D3 d) { return D3{(d.nx + 1) / 2, (d.ny + 1) / 2, (d.nz + 1) / 2}; }
long long vox(D3 d) { return (long long)d.nx * d.ny * d.nz; }

template <int MODE>
cudaError_t conv16(const __nv_bfloat16* in, D3 din, __nv_bfloat16* out, D3 dout, const __nv_bfloat16* W,
                   const float* bias, const __nv_bfloat16* skip, int relu, cudaStream_t s)
{
    const int xstep = MODE == CONVT_S2 ? 2 : 1;
    const int per_class = MODE == CONVT_S2 ? (dout.nx + 1) / 2 : dout.nx;
    const long long tiles = (long long)((per_class + 15) / 16) * xstep * dout.ny * dout.nz;
    k_conv16<MODE><<<(unsigned)((tiles + 3) / 4), 128, 0, s>>>(in, din, out, dout, W, bias, skip, relu);
    return cudaGetLastError();
}

int prep_weights(bsk_net* N)
{
    const int n = KT * C * C;
    k_prep_weights<<<blocks_for(n, 256), 256, 0, N->stream>>>(N->params + OFF_W2, N->w2, N->w2t, nullptr);
    k_prep_weights<<<blocks_for(n, 256), 256, 0, N->stream>>>(N->params + OFF_W3, N->w3, nullptr, N->w3f);
    k_prep_weights<<<blocks_for(n, 256), 256, 0, N->stream>>>(N->params + OFF_W4, N->w4, N->w4t, nullptr);
    k_round_bf16<<<blocks_for(NPARAM, 256), 256, 0, N->stream>>>(N->params, N->w_round, NPARAM);
    NCUDA(cudaGetLastError());
    return BSK_OK;
}

int forward(bsk_net* N, const float* r, const uint8_t* mask, float* z)
{
    const float* P = N->params;
    const float* R = N->w_round;
    const int relu = !N->linear;
    auto bias = [&](int off) -> const float* { return N->linear ? nullptr : P + off; };
    k_down1<<<blocks_for(vox(N->d1), 128), 128, 0, N->stream>>>(r, N->d0, N->a1, N->d1, R + OFF_W1, bias(OFF_B1),
                                                                relu);
    NCUDA(cudaGetLastError());
    NCUDA(conv16<CONV_S2>(N->a1, N->d1, N->a2, N->d2, N->w2, bias(OFF_B2), nullptr, relu, N->stream));
    NCUDA(conv16<CONV_S1>(N->a2, N->d2, N->a3, N->d2, N->w3, bias(OFF_B3), nullptr, relu, N->stream));
    NCUDA(conv16<CONVT_S2>(N->a3, N->d2, N->a4, N->d1, N->w4, bias(OFF_B4), N->a1, relu, N->stream));
    k_up1b<<<blocks_for(vox(N->d1), 128), 128, 0, N->stream>>>(N->a4, N->d1, z, N->d0, R + OFF_W5, bias(OFF_B5),
                                                               mask, r, P + OFF_WF);
    NCUDA(cudaGetLastError());
    return BSK_OK;
}

}  // namespace

extern "C" void bsk_net_destroy(bsk_net* N);

extern "C" int bsk_net_param_count(void) { return NPARAM; }

extern "C" int bsk_net_create(int nx, int ny, int nz, void* stream, bsk_net** out)
{
    if (!out || nx < 2 || ny < 2 || nz < 2) return nfail(BSK_EINVAL, "bad network grid");
    *out = nullptr;
    bsk_net* N = new (std::nothrow) bsk_net;
    if (!N) return nfail(BSK_ENOMEM, "host allocation failed");
    memset(N, 0, sizeof *N);
    N->d0 = D3{nx, ny, nz};
    N->d1 = halfdims(N->d0);
    N->d2 = halfdims(N->d1);
    N->stream = (cudaStream_t)stream;
    const long long v0 = vox(N->d0), v1 = vox(N->d1), v2 = vox(N->d2);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, N->stream);
    };
    for (float** p : {&N->params, &N->grad, &N->adam_m, &N->adam_v, &N->w_round})
        alloc((void**)p, NPARAM * sizeof(float));
    for (__nv_bfloat16** p : {&N->w2, &N->w3, &N->w4, &N->w2t, &N->w3f, &N->w4t})
        alloc((void**)p, KT * C * C * sizeof(__nv_bfloat16));
    alloc((void**)&N->a1, v1 * C * 2);
    alloc((void**)&N->a4, v1 * C * 2);
    alloc((void**)&N->g1, v1 * C * 2);
    alloc((void**)&N->g4, v1 * C * 2);
    alloc((void**)&N->a2, v2 * C * 2);
    alloc((void**)&N->a3, v2 * C * 2);
    alloc((void**)&N->g2, v2 * C * 2);
    alloc((void**)&N->g3, v2 * C * 2);
    alloc((void**)&N->z, v0 * sizeof(float));
    alloc((void**)&N->dz, v0 * sizeof(float));
    alloc((void**)&N->loss, sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        bsk_net_destroy(N);
        return nfail(BSK_ENOMEM, "network allocation failed");
    }
    *out = N;
    return BSK_OK;
}

extern "C" void bsk_net_destroy(bsk_net* N)
{
    if (!N) return;
    cudaStreamSynchronize(N->stream);
    void* ptrs[] = {N->params, N->grad, N->adam_m, N->adam_v, N->w_round, N->w2, N->w3, N->w4, N->w2t,
                    N->w3f, N->w4t, N->a1, N->a2, N->a3, N->a4, N->g1, N->g2, N->g3, N->g4, N->z, N->dz,
                    N->loss};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete N;
}

extern "C" int bsk_net_set_params(bsk_net* N, const float* params)
{
    if (!N || !params) return nfail(BSK_EINVAL, "null argument");
    NCUDA(cudaMemcpyAsync(N->params, params, NPARAM * sizeof(float), cudaMemcpyDefault, N->stream));
    NCUDA(cudaMemsetAsync(N->adam_m, 0, NPARAM * sizeof(float), N->stream));
    NCUDA(cudaMemsetAsync(N->adam_v, 0, NPARAM * sizeof(float), N->stream));
    N->adam_t = 0;
    return prep_weights(N);
}

extern "C" int bsk_net_set_activation(bsk_net* N, int act)
{
    if (!N || (act != BSK_ACT_RELU && act != BSK_ACT_LINEAR)) return nfail(BSK_EINVAL, "bad activation");
    N->linear = act == BSK_ACT_LINEAR;
    return BSK_OK;
}

namespace bsk {
bool net_linear(const bsk_net* N) { return N && N->linear; }
}  // namespace bsk

extern "C" int bsk_net_get_params(bsk_net* N, float* params)
{
    if (!N || !params) return nfail(BSK_EINVAL, "null argument");
    NCUDA(cudaMemcpyAsync(params, N->params, NPARAM * sizeof(float), cudaMemcpyDefault, N->stream));
    NCUDA(cudaStreamSynchronize(N->stream));
    return BSK_OK;
}

extern "C" int bsk_net_forward(bsk_net* N, const float* r, const uint8_t* mask, float* z)
{
    if (!N || !r || !z) return nfail(BSK_EINVAL, "null argument");
    return forward(N, r, mask, z);
}

extern "C" int bsk_net_zero_grad(bsk_net* N)
{
    if (!N) return nfail(BSK_EINVAL, "null network");
    NCUDA(cudaMemsetAsync(N->grad, 0, NPARAM * sizeof(float), N->stream));
    NCUDA(cudaMemsetAsync(N->loss, 0, sizeof(float), N->stream));
    return BSK_OK;
}

// Forward + backward of one sample; gradients accumulate into the network's gradient buffer.
namespace {

// Backward pass from the output gradient in N->dz (b5's gradient already added), activations
// of the forward pass of r in place.
int backward_from_dz(bsk_net* N, const float* r)
{
    const long long v0 = vox(N->d0), v1 = vox(N->d1), v2 = vox(N->d2);
    float* G = N->grad;
    const float* R = N->w_round;
    cudaStream_t s = N->stream;
    const int relu = !N->linear;
    auto relu_bwd = [&](__nv_bfloat16* g, const __nv_bfloat16* a, long long n, __nv_bfloat16* skip) {
        if (relu || skip)
            k_relu_bwd<<<std::min<long long>(blocks_for(n, 256), 4096), 256, 0, s>>>(g, a, n, skip, relu);
    };
    auto bias_grad = [&](const __nv_bfloat16* g, long long nv, int off) {
        if (relu) k_bias_grad16<<<256, 256, 0, s>>>(g, nv, G + off);   // linear: biases stay zero
    };
    k_wgrad1<<<blocks_for(v1, 64), 448, 0, s>>>(N->a4, N->d1, N->dz, N->d0, G + OFF_W5, 64);
    k_wgrad_fine<<<std::min<long long>(blocks_for(v0, 128), 512), 128, 0, s>>>(N->dz, r, N->d0, G + OFF_WF);
    // d a4 = down(dz; W5) (the adjoint of the transposed output convolution), then relu mask
    // (none for linear activations);
    // the skip connection passes the same gradient to a1
    k_down1<<<blocks_for(v1, 128), 128, 0, s>>>(N->dz, N->d0, N->g4, N->d1, R + OFF_W5, nullptr, 0);
    NCUDA(cudaMemsetAsync(N->g1, 0, v1 * C * 2, s));
    relu_bwd(N->g4, N->a4, v1 * C, N->g1);
    bias_grad(N->g4, v1, OFF_B4);
    k_wgrad16<CONVT_S2><<<blocks_for(v1, 256), 256, 0, s>>>(N->a3, N->d2, N->g4, N->d1, G + OFF_W4, 256);
    NCUDA(conv16<CONV_S2>(N->g4, N->d1, N->g3, N->d2, N->w4t, nullptr, nullptr, 0, s));
    // middle layer
    relu_bwd(N->g3, N->a3, v2 * C, nullptr);
    bias_grad(N->g3, v2, OFF_B3);
    k_wgrad16<CONV_S1><<<blocks_for(v2, 256), 256, 0, s>>>(N->a2, N->d2, N->g3, N->d2, G + OFF_W3, 256);
    NCUDA(conv16<CONV_S1>(N->g3, N->d2, N->g2, N->d2, N->w3f, nullptr, nullptr, 0, s));
    // second layer
    relu_bwd(N->g2, N->a2, v2 * C, nullptr);
    bias_grad(N->g2, v2, OFF_B2);
    k_wgrad16<CONV_S2><<<blocks_for(v2, 256), 256, 0, s>>>(N->a1, N->d1, N->g2, N->d2, G + OFF_W2, 256);
    // first layer: its gradient is the skip gradient plus convT(g2; W2^T), masked by a1 > 0
    // (g4 is free again and serves as the L1-sized buffer)
    NCUDA(conv16<CONVT_S2>(N->g2, N->d2, N->g4, N->d1, N->w2t, nullptr, N->g1, 0, s));
    relu_bwd(N->g4, N->a1, v1 * C, nullptr);
    bias_grad(N->g4, v1, OFF_B1);
    k_wgrad1<<<blocks_for(v1, 64), 448, 0, s>>>(N->g4, N->d1, r, N->d0, G + OFF_W1, 64);
    NCUDA(cudaGetLastError());
    return BSK_OK;
}

}  // namespace

extern "C" int bsk_net_backward(bsk_net* N, const float* r, const float* e, const uint8_t* mask,
                                float loss_weight)
{
    if (!N || !r || !e) return nfail(BSK_EINVAL, "null argument");
    if (int rc = forward(N, r, mask, N->z)) return rc;
    const long long v0 = vox(N->d0);
    k_loss<<<std::min<long long>(blocks_for(v0, 256), 1024), 256, 0, N->stream>>>(
        N->z, e, mask, v0, loss_weight, N->dz, N->loss, N->linear ? nullptr : N->grad + OFF_B5);
    NCUDA(cudaGetLastError());
    return backward_from_dz(N, r);
}

extern "C" int bsk_net_backward_grad(bsk_net* N, const float* r, const float* dz, const uint8_t* mask,
                                     float scale)
{
    if (!N || !r || !dz) return nfail(BSK_EINVAL, "null argument");
    if (int rc = forward(N, r, mask, N->z)) return rc;
    const long long v0 = vox(N->d0);
    k_given_grad<<<std::min<long long>(blocks_for(v0, 256), 1024), 256, 0, N->stream>>>(
        dz, mask, v0, scale, N->dz, N->linear ? nullptr : N->grad + OFF_B5);
    NCUDA(cudaGetLastError());
    return backward_from_dz(N, r);
}

extern "C" int bsk_net_adam(bsk_net* N, float lr, float scale)
{
    if (!N) return nfail(BSK_EINVAL, "null network");
    N->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - powf(b1, (float)N->adam_t), bc2 = 1.f - powf(b2, (float)N->adam_t);
    k_adam<<<blocks_for(NPARAM, 256), 256, 0, N->stream>>>(N->params, N->adam_m, N->adam_v, N->grad, NPARAM, lr, b1,
                                                          b2, 1e-8f, bc1, bc2, scale);
    NCUDA(cudaGetLastError());
    return prep_weights(N);
}

extern "C" int bsk_net_read_loss(bsk_net* N, float* loss, float* grad_out)
{
    if (!N || !loss) return nfail(BSK_EINVAL, "null argument");
    NCUDA(cudaMemcpyAsync(loss, N->loss, sizeof(float), cudaMemcpyDeviceToHost, N->stream));
    if (grad_out)
        NCUDA(cudaMemcpyAsync(grad_out, N->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, N->stream));
    NCUDA(cudaStreamSynchronize(N->stream));
    return BSK_OK;
}

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
// convolutions run on the 5th-generation tensor cores (tcgen05.mma, BF16 operands in shared
// memory, FP32 accumulator in tensor memory; an implicit GEMM over the 27 taps); the 1-channel
// ends and the weight gradients run on the FP32 pipes. The paper has no
// learned component: this is the workload's addition to the CG stage of section 2.5.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include <cuda_bf16.h>

#include "bsk.h"
#include "bsk_launch.h"
#include "tma_util.cuh"
#include "umma_util.cuh"

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

// ---- 16 -> 16 convolution on the 5th-generation tensor cores ----------------------------------
// out[o][co] = act( sum_{taps k, ci} W[k][co][ci] in[src(o,k)][ci] + bias[co] + skip[o][co] )
// as an implicit GEMM on tcgen05. A tile is 128 outputs of one output row (z, y), at x indices
// j0 .. j0 + 127 (for the transposed convolution, the outputs 2j and 2j + 1 for the same j, two
// accumulators), and
//   D[128][16] = sum over the tile's taps k of A_k[128][16] W_k^T,
// with D in tensor memory (FP32), one M = 128, N = 16, K = 16 BF16 MMA per tap. A_k is never
// gathered: along x the sources of consecutive outputs are consecutive voxels of one staged
// "plane" (S1: the source row; S2: its even or its odd voxels; transposed: the source row), so
// A_k is a plane seen from a start offset (the descriptor's start address). A plane holds 130
// voxels as two 8-channel halves, [half][slot] with 16 bytes per slot: the K-major no-swizzle
// operand layout (8 slots = one 128-byte core matrix, LBO = one half-plane, SBO = 128 bytes).
// The weights sit in shared memory as [tap][half][co][8 ci] (LBO 256, SBO 128).
// Per tile, one thread loads every half-plane the tile needs with a 4-D TMA box (the
// activation seen as [row][x][half][8 channels], x-stride 32 bytes, or 64 bytes for the even and
// odd voxels of S2; x neighbours outside the row arrive as zeros), all in flight at once on one
// mbarrier; it then issues the tile's MMAs and commits them to a second mbarrier, and warp w
// reads accumulator lanes 32w .. 32w + 31 (its outputs) for the epilogue. Several CTAs per SM
// overlap one another's phases.
constexpr int TC_M = 128;                  // outputs per tile (MMA M)
constexpr int TC_SLOTS = TC_M + 2;         // voxels per plane: the tile and its x halo
constexpr int TC_BOX = TC_SLOTS * 16;      // bytes one TMA box brings (one half-plane)
constexpr int TC_HALF = 2176;              // half-plane stride: TC_BOX rounded up to 128 bytes
constexpr int TC_PLANE = 2 * TC_HALF;
constexpr int TC_WTAP = 2 * C * 16;        // bytes of one tap's weights
constexpr uint32_t TC_COLS = 32;           // TMEM columns allocated (one or two 16-column accumulators)
constexpr uint64_t TC_WAIT_NS = 2000000000ull;

template <int MODE>
struct TcConv {
    // planes: S1 one per source row (kz, ky); S2 an even and an odd one per row; the transposed
    // convolution has at most 2 x 2 source rows, kept in (kz, ky) order
    static constexpr int PLANES = MODE == CONV_S2 ? 18 : MODE == CONV_S1 ? 9 : 4;
    static constexpr int IN_OFF = KT * TC_WTAP;
    static constexpr int BAR_OFF = IN_OFF + PLANES * TC_PLANE;
    static constexpr int SMEM = BAR_OFF + 32;   // two mbarriers and the TMEM address
};

struct ConvMaps {
    CUtensorMap m[2];
};

struct ConvArgs {
    CUtensorMap tin;        // the source activation (S2: its even voxels)
    CUtensorMap tin_odd;    // S2: its odd voxels
    D3 din, dout;
    __nv_bfloat16* out;
    const __nv_bfloat16* W;
    const float* bias;
    const __nv_bfloat16* skip;
    int relu;
    int* err;
};

template <int MODE>
__global__ void __launch_bounds__(128) k_conv16(const __grid_constant__ ConvArgs a)
{
    using L = TcConv<MODE>;
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    uint8_t* sw = tc_smem;
    uint8_t* sin = tc_smem + L::IN_OFF;
    uint64_t* full = reinterpret_cast<uint64_t*>(tc_smem + L::BAR_OFF);
    uint64_t* mma_done = full + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_smem + L::BAR_OFF + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const D3 din = a.din, dout = a.dout;

    // weights: global [k][co][16 ci] -> shared [k][half][co][8 ci], one 16-byte piece per step
    const uint4* Wg = reinterpret_cast<const uint4*>(a.W);
    for (int i = tid; i < KT * C * 2; i += blockDim.x) {
        const int h = i & 1, co = (i >> 1) % C, k = i / (2 * C);
        *reinterpret_cast<uint4*>(sw + k * TC_WTAP + h * (C * 16) + co * 16) = Wg[i];
    }
    if (warp == 0) bsk::tmem_alloc_warp(tslot, TC_COLS);
    if (tid == 32) {
        bsk::mbar_init(full, 1);
        bsk::mbar_init(mma_done, 1);
        bsk::fence_mbar_init();
        bsk::prefetch_tensormap(&a.tin);
        if (MODE == CONV_S2) bsk::prefetch_tensormap(&a.tin_odd);
    }
    bsk::fence_proxy_async_smem();
    bsk::tc_fence_before_sync();
    __syncthreads();
    bsk::tc_fence_after_sync();
    const uint32_t tmem = *tslot;

    const int per_class = MODE == CONVT_S2 ? (dout.nx + 1) / 2 : dout.nx;
    const int segs = (per_class + TC_M - 1) / TC_M;
    const long long ntiles = (long long)segs * dout.ny * dout.nz;
    const uint32_t idesc = bsk::umma_idesc_bf16_f32(TC_M, C);
    const uint32_t sin_a = bsk::smem_u32(sin), sw_a = bsk::smem_u32(sw);
    uint32_t phase = 0;
    int failed = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int seg = (int)(tile % segs);
        const long long row = tile / segs;
        const int oy = (int)(row % dout.ny), oz = (int)(row / dout.ny);
        const int j0 = seg * TC_M;
        int rows = 0;   // bit kz * 3 + ky: source row (kz, ky) exists
        for (int r = 0; r < 9; r++)
            if (src_index(MODE, oz, r / 3, din.nz) >= 0 && src_index(MODE, oy, r % 3, din.ny) >= 0)
                rows |= 1 << r;
        if (tid == 0) {
            const int per_row = MODE == CONV_S2 ? 4 : 2;
            bsk::mbar_arrive_expect_tx(full, (uint32_t)(__popc(rows) * per_row * TC_BOX));
            int q = 0;   // plane of the next source row (compacted for the transposed convolution)
            for (int r = 0; r < 9; r++) {
                if (!((rows >> r) & 1)) continue;
                const int srow = src_index(MODE, oz, r / 3, din.nz) * din.ny + src_index(MODE, oy, r % 3, din.ny);
                const int pl = MODE == CONV_S2 ? 2 * r : MODE == CONV_S1 ? r : q;
                const int x0 = MODE == CONV_S1 ? j0 - 1 : j0;
                for (int h = 0; h < 2; h++) {
                    bsk::tma_load_4d(sin + pl * TC_PLANE + h * TC_HALF, &a.tin, full, 0, h, x0, srow);
                    if (MODE == CONV_S2)   // odd voxels 2 (j0 + s) - 1 = 2 (j0 - 1 + s) + 1
                        bsk::tma_load_4d(sin + (pl + 1) * TC_PLANE + h * TC_HALF, &a.tin_odd, full, 0, h, j0 - 1, srow);
                }
                q++;
            }
        }
        // this thread's outputs: j; for the transposed convolution x = 2j and 2j + 1
        const int j = j0 + 32 * warp + lane;
        const int ox = MODE == CONVT_S2 ? 2 * j : j;
        const bool mine0 = ox < dout.nx;
        const bool mine1 = MODE == CONVT_S2 && ox + 1 < dout.nx;
        const long long o = ((long long)oz * dout.ny + oy) * dout.nx + ox;
        uint4 sk[4] = {};
        if (a.skip) {   // fetched while the tile's loads and MMAs run
            const uint4* sp = reinterpret_cast<const uint4*>(a.skip + o * C);
            if (mine0) { sk[0] = sp[0]; sk[1] = sp[1]; }
            if (mine1) { sk[2] = sp[2]; sk[3] = sp[3]; }
        }
        int bad = 0;
        if (tid == 0) {
            const bool landed = bsk::mbar_wait_bounded(full, phase, TC_WAIT_NS);
            if (!landed) bad = 1;   // no MMAs on a tile whose loads did not land
            bsk::tc_fence_after_sync();
            uint32_t acc0 = 0, acc1 = 0;
            int q = 0;
            for (int r = 0; landed && r < 9; r++) {
                if (!((rows >> r) & 1)) continue;
                const uint32_t pbase = sin_a + (uint32_t)((MODE == CONV_S2 ? 2 * r : MODE == CONV_S1 ? r : q) * TC_PLANE);
                for (int kx = 0; kx < 3; kx++) {
                    // plane offset and start slot of tap kx (see the layout above)
                    uint32_t off;
                    if (MODE == CONV_S1) off = kx * 16;
                    else if (MODE == CONV_S2) off = kx == 1 ? 0 : TC_PLANE + (kx == 2 ? 16 : 0);
                    else off = kx == 0 ? 16 : 0;   // kx = 1 feeds x = 2j, kx = 0 and 2 feed 2j + 1
                    const uint64_t ad = bsk::umma_desc_noswizzle(pbase + off, TC_HALF, 128);
                    const uint64_t bd = bsk::umma_desc_noswizzle(sw_a + (uint32_t)((r * 3 + kx) * TC_WTAP), C * 16, 128);
                    if (MODE == CONVT_S2 && kx != 1) {
                        bsk::umma_bf16(tmem + 16, ad, bd, idesc, acc1);
                        acc1 = 1;
                    } else {
                        bsk::umma_bf16(tmem, ad, bd, idesc, acc0);
                        acc0 = 1;
                    }
                }
                q++;
            }
            bsk::umma_commit(mma_done);   // arrives when the MMAs issued above are done
        }
        if (!bsk::mbar_wait_bounded(mma_done, phase, TC_WAIT_NS)) bad = 1;
        phase ^= 1;
        __nv_bfloat16* dst = a.out + o * C;
        if (__syncthreads_or(bad)) {
            // a load or the MMAs did not complete in time: mark this tile's outputs NaN, report, stop
            const uint4 nan4 = make_uint4(0x7FC07FC0u, 0x7FC07FC0u, 0x7FC07FC0u, 0x7FC07FC0u);
            uint4* d4 = reinterpret_cast<uint4*>(dst);
            if (mine0) { d4[0] = nan4; d4[1] = nan4; }
            if (mine1) { d4[2] = nan4; d4[3] = nan4; }
            failed = 1;
            break;
        }
        bsk::tc_fence_after_sync();
#pragma unroll
        for (int par = 0; par < (MODE == CONVT_S2 ? 2 : 1); par++) {
            uint32_t v[16];
            bsk::tmem_ld_32x32b_x16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * par, v);
            if (!(par ? mine1 : mine0)) continue;
            float f[C];
#pragma unroll
            for (int c = 0; c < C; c++) f[c] = __uint_as_float(v[c]) + (a.bias ? a.bias[c] : 0.f);
            if (a.skip) {
                const uint32_t sv[8] = {sk[2 * par].x, sk[2 * par].y, sk[2 * par].z, sk[2 * par].w,
                                        sk[2 * par + 1].x, sk[2 * par + 1].y, sk[2 * par + 1].z, sk[2 * par + 1].w};
#pragma unroll
                for (int c = 0; c < C / 2; c++) {
                    const float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&sv[c]));
                    f[2 * c] += t.x;
                    f[2 * c + 1] += t.y;
                }
            }
            uint32_t w[C / 2];
#pragma unroll
            for (int c = 0; c < C / 2; c++) {
                float x0 = f[2 * c], x1 = f[2 * c + 1];
                if (a.relu) { x0 = fmaxf(x0, 0.f); x1 = fmaxf(x1, 0.f); }
                const __nv_bfloat162 hv = __floats2bfloat162_rn(x0, x1);
                w[c] = *reinterpret_cast<const uint32_t*>(&hv);
            }
            uint4* d4 = reinterpret_cast<uint4*>(dst) + 2 * par;
            d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
            d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
        bsk::tc_fence_before_sync();
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) atomicExch(a.err, 1);
        // let the loads and MMAs in flight finish (bounded) before the CTA's memory goes away
        bsk::mbar_wait_bounded(full, phase ^ 1u, TC_WAIT_NS);
        bsk::mbar_wait_bounded(mma_done, phase ^ 1u, TC_WAIT_NS);
    }
    bsk::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        bsk::tc_fence_after_sync();
        bsk::tmem_dealloc_warp(tmem, TC_COLS);
    }
}

// ---- 1-channel ends (FP32 pipes) ----------------------------------------------------------
// out[o][c] = act( sum_k W[k][c] x[2o + k - 1] + bias[c] ), x fine (FP32, 1 channel), out coarse.
// One thread per coarse output; the grid is (x blocks, coarse y, coarse z), so no index is
// decoded by division. Channel pairs accumulate in packed f32x2 FMAs (the same roundings as
// scalar FMAs, in the same order).
__global__ void __launch_bounds__(128) k_down1(const float* __restrict__ x, D3 din, __nv_bfloat16* __restrict__ out, D3 dout,
                        const float* __restrict__ W, const float* __restrict__ bias, int relu)
{
    __shared__ float2 sW[KT * C / 2];
    for (int i = threadIdx.x; i < KT * C / 2; i += blockDim.x) sW[i] = make_float2(W[2 * i], W[2 * i + 1]);
    __syncthreads();
    const int ox = blockIdx.x * blockDim.x + threadIdx.x, oy = blockIdx.y, oz = blockIdx.z;
    if (ox >= dout.nx) return;
    float2 acc[C / 2];
#pragma unroll
    for (int c = 0; c < C / 2; c++) acc[c] = bias ? make_float2(bias[2 * c], bias[2 * c + 1]) : make_float2(0.f, 0.f);
    const int ix = 2 * ox;   // <= din.nx - 1: the coarse grid is the fine one halved, rounded up
    for (int kz = 0; kz < 3; kz++) {
        const int iz = 2 * oz + kz - 1;
        if (iz < 0 || iz >= din.nz) continue;
        for (int ky = 0; ky < 3; ky++) {
            const int iy = 2 * oy + ky - 1;
            if (iy < 0 || iy >= din.ny) continue;
            const float* row = x + ((long long)iz * din.ny + iy) * din.nx;
            const float v[3] = {ix >= 1 ? row[ix - 1] : 0.f, row[ix], ix + 1 < din.nx ? row[ix + 1] : 0.f};
#pragma unroll
            for (int kx = 0; kx < 3; kx++) {
                const float2 vv = make_float2(v[kx], v[kx]);
                const float2* w = sW + ((kz * 3 + ky) * 3 + kx) * (C / 2);
#pragma unroll
                for (int c = 0; c < C / 2; c++) acc[c] = __ffma2_rn(w[c], vv, acc[c]);
            }
        }
    }
    uint32_t w[C / 2];   // the voxel's 16 channels, stored as two 16-byte vectors
#pragma unroll
    for (int c = 0; c < C / 2; c++) {
        float v0 = acc[c].x, v1 = acc[c].y;
        if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        w[c] = *reinterpret_cast<const uint32_t*>(&h);
    }
    uint4* dst = reinterpret_cast<uint4*>(out + (((long long)oz * dout.ny + oy) * dout.nx + ox) * C);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// Output layer, z[o] = mask * ( sum_{k valid} sum_c W[k][c] a[srcT(o,k)][c] + b
//                                 + sum_k Wf[k] r[o + k - 1] ), a coarse (BF16), z and r fine.
// One thread per 2 x 2 x 2 block of fine voxels (2m .. 2m+1 per axis), which gathers from the
// 2 x 2 x 2 coarse voxels m .. m+1, so that each coarse voxel is loaded once for the eight
// outputs it feeds. Along an axis, fine 2m + e takes coarse m + d with tap k = e + 1 - 2d (the
// transposed stride-2 gather of src_index: (e, d) = (0, 0) -> 1, (1, 0) -> 2, (1, 1) -> 0,
// (0, 1) none). The full-resolution filter of the eight outputs reads the 4 x 4 x 4 patch of r
// around the block (fine 2m - 1 .. 2m + 2 per axis, zeros outside the grid) once, one z-plane at
// a time. The grid is (x blocks, coarse y, coarse z), so no index is decoded by division.
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
    const int mx = blockIdx.x * blockDim.x + threadIdx.x, my = blockIdx.y, mz = blockIdx.z;
    if (mx >= din.nx) return;
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
    // the full-resolution filter of r: the 4 x 4 x 4 patch around the block (fine 2m - 1 .. 2m + 2
    // per axis, zeros outside the grid), one z-plane of it at a time; plane i feeds the outputs
    // with ez + kz = i, so each output still adds its taps in (kz, ky, kx) order
    float fine[8];
#pragma unroll
    for (int e = 0; e < 8; e++) fine[e] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int fz = 2 * mz - 1 + i;
        float p[4][4];   // r at fine (fz, 2my - 1 + j, 2mx - 1 + l)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int fy = 2 * my - 1 + j;
            const bool rowok = fz >= 0 && fz < dout.nz && fy >= 0 && fy < dout.ny;
            const float* rr = r + ((long long)(rowok ? fz : 0) * dout.ny + (rowok ? fy : 0)) * dout.nx;
#pragma unroll
            for (int l = 0; l < 4; l++) {
                const int fx = 2 * mx - 1 + l;
                p[j][l] = rowok && fx >= 0 && fx < dout.nx ? rr[fx] : 0.f;
            }
        }
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int ez = e >> 2, ey = (e >> 1) & 1, ex = e & 1;
            const int kz = i - ez;
            if (kz < 0 || kz > 2 || !(act & (1 << e))) continue;
#pragma unroll
            for (int ky = 0; ky < 3; ky++)
#pragma unroll
                for (int kx = 0; kx < 3; kx++)
                    fine[e] = fmaf(sF[(kz * 3 + ky) * 3 + kx], p[ey + ky][ex + kx], fine[e]);
        }
    }
    const float b5 = bias ? bias[0] : 0.f;
#pragma unroll
    for (int e = 0; e < 8; e++) {
        if (!(act & (1 << e))) continue;
        const int fz = 2 * mz + (e >> 2), fy = 2 * my + ((e >> 1) & 1), fx = 2 * mx + (e & 1);
        z[((long long)fz * dout.ny + fy) * dout.nx + fx] = acc[e] + b5 + fine[e];
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

// Grid of the 1-channel end kernels: 128-thread blocks along x, one per coarse (y, z) row.
dim3 grid_xyz(D3 d) { return dim3((unsigned)((d.nx + 127) / 128), (unsigned)d.ny, (unsigned)d.nz); }

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
    int* tc_err;                                 // set by a convolution whose loads or MMAs timed out
    void* tc_zero;                               // 64 zero bytes (conv_maps)
    ConvMaps map_a1, map_a2, map_a3;             // sources of the forward convolutions
    ConvMaps map_g4, map_g3, map_g2;             // sources of the backward (input-gradient) ones
    int adam_t;
    int linear;                                  // BSK_ACT_LINEAR: identity activations, no biases
};

namespace {

int nfail(int code, const char* msg) { return bsk::set_error(code, msg); }

// After a synchronisation of the network's stream: BSK_ETIMEOUT if a convolution's MMAs did not
// complete within its bounded wait (its outputs were then set to NaN), else BSK_OK.
int tc_status(bsk_net* N)
{
    int flag = 0;
    if (cudaMemcpy(&flag, N->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return nfail(BSK_ECUDA, "reading the network's error word failed");
    return flag ? nfail(BSK_ETIMEOUT, "a network convolution's tensor-core wait timed out") : BSK_OK;
}

#define NCUDA(call)                                                        \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return nfail(BSK_ECUDA, #call " failed");   \
    } while (0)

D3 halfdims(D3 d) { return D3{(d.nx + 1) / 2, (d.ny + 1) / 2, (d.nz + 1) / 2}; }
long long vox(D3 d) { return (long long)d.nx * d.ny * d.nz; }

// Persistent launch: as many CTAs as fit on the SMs (shared memory decides: 4 per SM for S1, 2
// for S2, 7 for the transposed convolution; their TMEM columns, 32 each, always fit in the 512),
// each looping over tiles. `maps` holds the source activation's tensor maps (see conv_maps).
template <int MODE>
cudaError_t conv16(const ConvMaps& maps, D3 din, __nv_bfloat16* out, D3 dout, const __nv_bfloat16* W,
                   const float* bias, const __nv_bfloat16* skip, int relu, int* err, cudaStream_t s)
{
    constexpr int smem = TcConv<MODE>::SMEM;
    int dev = 0, sms = 0, smem_sm = 0, reserved = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv16<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv16<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // CTAs the SM's shared memory holds (at most 16 of 128 threads; 16 x 32 TMEM columns fit)
    const int per_sm = std::max(1, std::min(16, smem_sm / (smem + reserved)));
    ConvArgs a;
    a.tin = maps.m[0];
    a.tin_odd = maps.m[1];
    a.din = din;
    a.dout = dout;
    a.out = out;
    a.W = W;
    a.bias = bias;
    a.skip = skip;
    a.relu = relu;
    a.err = err;
    const int per_class = MODE == CONVT_S2 ? (dout.nx + 1) / 2 : dout.nx;
    const long long tiles = (long long)((per_class + TC_M - 1) / TC_M) * dout.ny * dout.nz;
    const long long grid = std::min<long long>(tiles, (long long)sms * per_sm);
    k_conv16<MODE><<<(unsigned)grid, 128, smem, s>>>(a);
    return cudaGetLastError();
}

// Tensor maps of a BF16 channels-last activation of grid d, seen as the 4-D array
// [row = z * ny + y][x][half][8 channels]. A box is one half of 130 consecutive voxels of a row
// (8 channels x 1 half x 130 x 1 = 2080 bytes), which lands in shared memory as a half-plane.
// For a stride-2 source (S2) m[0] covers the even voxels and m[1] the odd ones (x-stride 64
// bytes; the odd map starts at voxel 1); `zero` (64 zero bytes) stands in for the odd voxels of a
// 1-voxel-wide grid.
int conv_maps(ConvMaps& cm, const __nv_bfloat16* base, D3 d, bool stride2, const void* zero)
{
    auto fn = bsk::tensor_map_encoder();
    if (!fn) return nfail(BSK_ECUDA, "cuTensorMapEncodeTiled is not available");
    auto enc = [&](CUtensorMap* m, const void* ptr, long long nx, long long xstride, long long rows,
                   long long rowstride) -> int {
        const cuuint64_t dims[4] = {8u, 2u, (cuuint64_t)nx, (cuuint64_t)rows};
        const cuuint64_t strides[3] = {16u, (cuuint64_t)xstride, (cuuint64_t)rowstride};
        const cuuint32_t box[4] = {8u, 1u, (cuuint32_t)TC_SLOTS, 1u};
        const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
        CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        return r == CUDA_SUCCESS ? BSK_OK : nfail(BSK_ECUDA, "network tensor map encoding failed");
    };
    const long long rows = (long long)d.ny * d.nz, rs = (long long)d.nx * C * 2;
    memset(&cm, 0, sizeof cm);
    if (!stride2) return enc(&cm.m[0], base, d.nx, 32, rows, rs);
    if (int rc = enc(&cm.m[0], base, (d.nx + 1) / 2, 64, rows, rs)) return rc;
    if (d.nx >= 2) return enc(&cm.m[1], base + C, d.nx / 2, 64, rows, rs);
    return enc(&cm.m[1], zero, 1, 64, 1, 64);
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
    k_down1<<<grid_xyz(N->d1), 128, 0, N->stream>>>(r, N->d0, N->a1, N->d1, R + OFF_W1, bias(OFF_B1),
                                                                relu);
    NCUDA(cudaGetLastError());
    NCUDA(conv16<CONV_S2>(N->map_a1, N->d1, N->a2, N->d2, N->w2, bias(OFF_B2), nullptr, relu, N->tc_err, N->stream));
    NCUDA(conv16<CONV_S1>(N->map_a2, N->d2, N->a3, N->d2, N->w3, bias(OFF_B3), nullptr, relu, N->tc_err, N->stream));
    NCUDA(conv16<CONVT_S2>(N->map_a3, N->d2, N->a4, N->d1, N->w4, bias(OFF_B4), N->a1, relu, N->tc_err,
                           N->stream));
    k_up1b<<<grid_xyz(N->d1), 128, 0, N->stream>>>(N->a4, N->d1, z, N->d0, R + OFF_W5, bias(OFF_B5),
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
    if (N->d1.ny > 65535 || N->d1.nz > 65535) {   // grid_xyz: one block row per coarse (y, z)
        delete N;
        return nfail(BSK_EINVAL, "network grid too large in y or z");
    }
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
    alloc((void**)&N->tc_err, sizeof(int));
    alloc(&N->tc_zero, 64);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bsk_net_destroy(N);
        return nfail(BSK_ENOMEM, "network allocation failed");
    }
    int rc = conv_maps(N->map_a1, N->a1, N->d1, true, N->tc_zero);
    if (!rc) rc = conv_maps(N->map_a2, N->a2, N->d2, false, N->tc_zero);
    if (!rc) rc = conv_maps(N->map_a3, N->a3, N->d2, false, N->tc_zero);
    if (!rc) rc = conv_maps(N->map_g4, N->g4, N->d1, true, N->tc_zero);
    if (!rc) rc = conv_maps(N->map_g3, N->g3, N->d2, false, N->tc_zero);
    if (!rc) rc = conv_maps(N->map_g2, N->g2, N->d2, false, N->tc_zero);
    if (rc) {
        bsk_net_destroy(N);
        return rc;
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
                    N->loss, N->tc_err, N->tc_zero};
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
    return tc_status(N);
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
    k_down1<<<grid_xyz(N->d1), 128, 0, s>>>(N->dz, N->d0, N->g4, N->d1, R + OFF_W5, nullptr, 0);
    NCUDA(cudaMemsetAsync(N->g1, 0, v1 * C * 2, s));
    relu_bwd(N->g4, N->a4, v1 * C, N->g1);
    bias_grad(N->g4, v1, OFF_B4);
    k_wgrad16<CONVT_S2><<<blocks_for(v1, 256), 256, 0, s>>>(N->a3, N->d2, N->g4, N->d1, G + OFF_W4, 256);
    NCUDA(conv16<CONV_S2>(N->map_g4, N->d1, N->g3, N->d2, N->w4t, nullptr, nullptr, 0, N->tc_err, s));
    // middle layer
    relu_bwd(N->g3, N->a3, v2 * C, nullptr);
    bias_grad(N->g3, v2, OFF_B3);
    k_wgrad16<CONV_S1><<<blocks_for(v2, 256), 256, 0, s>>>(N->a2, N->d2, N->g3, N->d2, G + OFF_W3, 256);
    NCUDA(conv16<CONV_S1>(N->map_g3, N->d2, N->g2, N->d2, N->w3f, nullptr, nullptr, 0, N->tc_err, s));
    // second layer
    relu_bwd(N->g2, N->a2, v2 * C, nullptr);
    bias_grad(N->g2, v2, OFF_B2);
    k_wgrad16<CONV_S2><<<blocks_for(v2, 256), 256, 0, s>>>(N->a1, N->d1, N->g2, N->d2, G + OFF_W2, 256);
    // first layer: its gradient is the skip gradient plus convT(g2; W2^T), masked by a1 > 0
    // (g4 is free again and serves as the L1-sized buffer)
    NCUDA(conv16<CONVT_S2>(N->map_g2, N->d2, N->g4, N->d1, N->w2t, nullptr, N->g1, 0, N->tc_err, s));
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
    return tc_status(N);
}

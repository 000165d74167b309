// tma_impl.cuh -- host launchers of the TMA operator kernel for one element type. Included once
// by tma_f32.cu (BSK_T = float), once by tma_f64.cu (BSK_T = double) and once by tma_df.cu
// (BSK_T = dfl, the double-float operator and residual; BSK_TMA_NO_CG).
#pragma once

#include <type_traits>

#include <cudaTypedefs.h>

#include "bsk_launch.h"
#include "op_tma.cuh"

namespace bsk {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() { return tensor_map_encoder(); }

// 3-D map of an [nz][ny][nx] array of T with box (bx, by, 1); out-of-range elements read as 0.
cudaError_t encode_box(CUtensorMap* m, const void* base, int nx, int ny, int nz, int bx, int by)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(BSK_T), (cuuint64_t)nx * ny * sizeof(BSK_T)};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = fn(m, sizeof(BSK_T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                    3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

#ifndef BSK_TMA_NO_CG
#define BSK_TMA_NO_CG 0
#endif

// kernel coefficient of the element type (double-float: split on the host)
template <typename U>
U coef_cast(double v)
{
    if constexpr (std::is_same<U, dfl>::value) return dfl::from_double_host(v);
    else return (U)v;
}

struct TmaInfo {
    bool ready = false;
    int grid = 0;   // resident blocks on the whole GPU
};

template <int N, int MODE>
TmaInfo& tma_info()
{
    static TmaInfo info;
    return info;
}

template <int N, int MODE>
cudaError_t prepare_one()
{
    TmaInfo& info = tma_info<N, MODE>();
    if (info.ready) return cudaSuccess;
    using LY = TLayout<BSK_T, N, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k_op_tma<BSK_T, N, MODE, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::total);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_op_tma<BSK_T, N, MODE, false>, kTNT, LY::total);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    info.grid = per_sm * sms;
    info.ready = true;
    return cudaSuccess;
}

template <int N>
cudaError_t prepare_degree_tma()
{
    cudaError_t e = prepare_one<N, TMODE_OP>();
    if constexpr (std::is_same<BSK_T, float>::value && N <= 4) {
        if (e == cudaSuccess) e = prepare_ws(N);
    }
    if (e == cudaSuccess) e = prepare_one<N, TMODE_RES>();
#if !BSK_TMA_NO_CG
    if (e == cudaSuccess) e = prepare_one<N, TMODE_CG>();
#endif
    return e;
}

// Items = tiles x z-chunks. Chooses the z-chunk count that minimises rounds x planes per item
// (halo planes included) for the resident grid, with chunks of at most kMaxChunk planes: the
// blocks of one wave of items drift apart in z as they march, and once neighbouring tiles are
// far apart their shared halo rows no longer meet in L2 (a whole-column item at 928^3 read
// 30 B/unknown from DRAM for 16 B of algorithmic reads; chunks of <= 128 planes cut the CG
// iteration from 6.65 to 5.98 ms on GB300).
constexpr int kMaxChunk = 128;

void plan(int nx, int ny, int nz, int n, int grid, int& tiles_x, int& tiles_y, int& tz, int& nitems)
{
    tiles_x = (nx + kTX - 1) / kTX;
    tiles_y = (ny + kTY - 1) / kTY;
    const long long tiles = (long long)tiles_x * tiles_y;
    long long best = -1;
    int best_tz = nz;
    for (int nzc = 1; nzc <= nz; nzc++) {
        const int t = (nz + nzc - 1) / nzc;
        if (t > kMaxChunk && t > 1) continue;
        if (best >= 0 && t < kMaxChunk / 4) break;   // no finer chunking than needed
        const int chunks = (nz + t - 1) / t;
        const long long items = tiles * chunks;
        const long long rounds = (items + grid - 1) / grid;
        const long long cost = rounds * (t + 2 * n);
        if (best < 0 || cost < best) { best = cost; best_tz = t; }
    }
    tz = best_tz;
    nitems = (int)(tiles * ((nz + tz - 1) / tz));
}

template <int N, int MODE>
cudaError_t launch_one(const TmaLaunch& L, cudaStream_t s)
{
    if constexpr (std::is_same<BSK_T, float>::value && (MODE == TMODE_OP || MODE == TMODE_CG) && N <= 4) {
        // the warp-specialised operator pass; for CG the one the handle's tuning chose
        if (!L.mask && !L.zpad && (MODE == TMODE_OP || L.impl == 0)) return launch_ws(L, s);
    }
    if (L.zpad && MODE != TMODE_OP) return cudaErrorInvalidValue;   // slabs: operator passes only
    const int nz_in = L.nz + 2 * L.zpad;                              // planes of the input array
    TmaInfo& info = tma_info<N, MODE>();
    if (!info.ready) return cudaErrorNotReady;   // prepare_tma was not called
    using G = TGeo<BSK_T, N>;
    using LY = TLayout<BSK_T, N, MODE>;
    TmaArgs<BSK_T> a;
    memset(&a, 0, sizeof a);
    cudaError_t e;
    const int nin = MODE == TMODE_CG ? 3 : 1;
    for (int i = 0; i < nin; i++)
        if ((e = encode_box(&a.tin[i], L.in[i], L.nx, L.ny, nz_in, G::BX, G::HY)) != cudaSuccess) return e;
    if (MODE != TMODE_OP)
        if ((e = encode_box(&a.tint, L.inint, L.nx, L.ny, L.nz, G::IP, kTY)) != cudaSuccess) return e;
    a.out0 = static_cast<BSK_T*>(L.out0);
    a.out1 = static_cast<BSK_T*>(L.out1);
    a.out2 = static_cast<BSK_T*>(L.out2);
    a.xvec = static_cast<BSK_T*>(L.xvec);
    if (L.mask && !L.mbits) return cudaErrorInvalidValue;   // the kernels read the packed mask
    a.mbits = L.mask ? L.mbits : nullptr;
    a.mwords = mask_words(L.nx);
    a.occ = L.mask ? L.occ : nullptr;
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.z_off = L.z_off;
    a.nz_glob = L.nz_glob > 0 ? L.nz_glob : L.nz;
    a.zpad = L.zpad;
    a.pitch = L.nx;
    plan(L.nx, L.ny, L.nz, N, info.grid, a.tiles_x, a.tiles_y, a.tz, a.nitems);
    for (int d = 0; d < 3; d++)
        for (int j = 0; j < kMaxTaps; j++) {
            a.M[d][j] = coef_cast<BSK_T>(L.M[d][j]);
            a.K[d][j] = coef_cast<BSK_T>(L.Kdt[d][j]);
        }
    a.sc = L.sc;
    a.partials = L.partials;
    a.work = L.work;
    a.fin = L.fin;
    const int grid = a.nitems < info.grid ? a.nitems : info.grid;
    k_op_tma<BSK_T, N, MODE, false><<<grid, kTNT, LY::total, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_degree(const TmaLaunch& L, cudaStream_t s)
{
    switch (L.mode) {
    case TMODE_OP: return launch_one<N, TMODE_OP>(L, s);
#if !BSK_TMA_NO_CG
    case TMODE_CG: return launch_one<N, TMODE_CG>(L, s);
#endif
    case TMODE_RES: return launch_one<N, TMODE_RES>(L, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <>
int tma_max_degree<BSK_T>()
{
    return sizeof(BSK_T) == 4 ? 5 : 3;
}

template <>
cudaError_t prepare_tma<BSK_T>(int degree)
{
    switch (degree) {
    case 1: return prepare_degree_tma<1>();
    case 2: return prepare_degree_tma<2>();
    case 3: return prepare_degree_tma<3>();
#if BSK_TMA_HIGH_DEGREE
    case 4: return prepare_degree_tma<4>();
    case 5: return prepare_degree_tma<5>();
#endif
    default: return cudaErrorInvalidValue;
    }
}

template <>
int tma_grid<BSK_T>(int degree, int mode)
{
    switch (degree * 4 + mode) {
#define BSK_G(N_, M_) case N_ * 4 + M_: return tma_info<N_, M_>().grid;
        BSK_G(1, TMODE_OP) BSK_G(1, TMODE_RES) BSK_G(1, TMODE_CG)
        BSK_G(2, TMODE_OP) BSK_G(2, TMODE_RES) BSK_G(2, TMODE_CG)
        BSK_G(3, TMODE_OP) BSK_G(3, TMODE_RES) BSK_G(3, TMODE_CG)
#if BSK_TMA_HIGH_DEGREE
        BSK_G(4, TMODE_OP) BSK_G(4, TMODE_RES) BSK_G(4, TMODE_CG)
        BSK_G(5, TMODE_OP) BSK_G(5, TMODE_RES) BSK_G(5, TMODE_CG)
#endif
#undef BSK_G
    default: return 0;
    }
}

template <>
cudaError_t launch_tma<BSK_T>(const TmaLaunch& L, cudaStream_t s)
{
    switch (L.degree) {
    case 1: return launch_degree<1>(L, s);
    case 2: return launch_degree<2>(L, s);
    case 3: return launch_degree<3>(L, s);
#if BSK_TMA_HIGH_DEGREE
    case 4: return launch_degree<4>(L, s);
    case 5: return launch_degree<5>(L, s);
#endif
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsk

// ws_f32.cu -- host launchers of the warp-specialised FP32 operator and CG passes (op_ws.cuh).
#include <cstring>

#include <cudaTypedefs.h>

#include "bsk_launch.h"
#include "op_ws.cuh"

namespace bsk {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 ws_encode_fn() { return tensor_map_encoder(); }

struct WsInfo {
    bool ready = false;
    int grid = 0;   // resident blocks on the whole GPU
};

template <int N, int MODE, bool ISO>
WsInfo& ws_info()
{
    static WsInfo info;
    return info;
}

template <int N, int MODE, bool ISO>
cudaError_t ws_prepare_k()
{
    WsInfo& info = ws_info<N, MODE, ISO>();
    if (info.ready) return cudaSuccess;
    using G = WsGeo<N, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k_ws<N, MODE, ISO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::total);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ws<N, MODE, ISO>, kWsNT, G::total);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    info.grid = per_sm * sms;
    info.ready = true;
    return cudaSuccess;
}

template <int N>
cudaError_t ws_prepare_n()
{
    cudaError_t e = ws_prepare_k<N, WS_OP, true>();
    if (e == cudaSuccess) e = ws_prepare_k<N, WS_OP, false>();
    if (e == cudaSuccess) e = ws_prepare_k<N, WS_CG, true>();
    if (e == cudaSuccess) e = ws_prepare_k<N, WS_CG, false>();
    return e;
}

// Items = tiles x z-chunks, handed out round-robin to the resident blocks. The chunk count
// minimises rounds x planes per item (2n halo planes included), with chunks of at most
// max_chunk planes. The cap trades two effects that the cost model does not see: short chunks
// keep the blocks working on neighbouring tiles close in z, so that their shared halo rows meet
// in L2; but they make many rounds, over which the blocks drift apart all the same. The CG pass
// takes the cap its handle's tuning chose (bsk_select_cg_kernel); the operator keeps 128.
constexpr int kWsDefaultChunk = 128;

void ws_plan(int nx, int ny, int nz, int n, int grid, int max_chunk, int& tiles_x, int& tiles_y, int& tz,
             int& nitems)
{
    const int kMaxChunk = max_chunk > 0 ? max_chunk : kWsDefaultChunk;
    tiles_x = (nx + kWsTX - 1) / kWsTX;
    tiles_y = (ny + kWsTY - 1) / kWsTY;
    const long long tiles = (long long)tiles_x * tiles_y;
    long long best = -1;
    int best_tz = nz;
    for (int nzc = 1; nzc <= nz; nzc++) {
        const int t = (nz + nzc - 1) / nzc;
        if (t > kMaxChunk && t > 1) continue;
        if (best >= 0 && t < kMaxChunk / 4) break;
        const long long items = tiles * ((nz + t - 1) / t);
        const long long rounds = (items + grid - 1) / grid;
        const long long cost = rounds * (t + 2 * n);
        if (best < 0 || cost < best) {
            best = cost;
            best_tz = t;
        }
    }
    tz = best_tz;
    nitems = (int)(tiles * ((nz + tz - 1) / tz));
}

cudaError_t ws_encode(CUtensorMap* m, const void* base, int nx, int ny, int nz, int bx, int by)
{
    auto fn = ws_encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Isotropic grid: the three axes' kernels coincide (then the y/z threads share tap sets).
bool ws_isotropic(const TmaLaunch& L)
{
    for (int j = 0; j < kMaxTaps; j++)
        if (L.M[0][j] != L.M[1][j] || L.M[1][j] != L.M[2][j] || L.Kdt[0][j] != L.Kdt[1][j] ||
            L.Kdt[1][j] != L.Kdt[2][j])
            return false;
    return true;
}

template <int N, int MODE, bool ISO>
cudaError_t ws_launch_k(const TmaLaunch& L, cudaStream_t s)
{
    WsInfo& info = ws_info<N, MODE, ISO>();
    if (!info.ready) return cudaErrorNotReady;   // prepare_ws was not called
    using G = WsGeo<N, MODE>;
    WsArgs a;
    memset(&a, 0, sizeof a);
    cudaError_t e;
    for (int i = 0; i < G::NIN; i++)
        if ((e = ws_encode(&a.tin[i], L.in[i], L.nx, L.ny, L.nz, G::BX, G::HY)) != cudaSuccess) return e;
    if (MODE == WS_CG)
        if ((e = ws_encode(&a.tint, L.inint, L.nx, L.ny, L.nz, G::IP, kWsTY)) != cudaSuccess) return e;
    a.out0 = static_cast<float*>(L.out0);
    a.out1 = static_cast<float*>(L.out1);
    a.out2 = static_cast<float*>(L.out2);
    a.xvec = static_cast<float*>(L.xvec);
    a.sc = L.sc;
    a.partials = L.partials;
    a.fin = MODE == WS_CG ? L.fin : FIN_NONE;
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    ws_plan(L.nx, L.ny, L.nz, N, info.grid, MODE == WS_CG ? L.ws_chunk : 0, a.tiles_x, a.tiles_y, a.tz,
            a.nitems);
    for (int d = 0; d < 3; d++)
        for (int j = 0; j < kMaxTaps; j++) {
            a.M[d][j] = (float)L.M[d][j];
            a.K[d][j] = (float)L.Kdt[d][j];
        }
    const int grid = a.nitems < info.grid ? a.nitems : info.grid;
    k_ws<N, MODE, ISO><<<grid, kWsNT, G::total, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t ws_launch_n(const TmaLaunch& L, cudaStream_t s)
{
    const bool iso = ws_isotropic(L);
    if (L.mode == TMODE_OP) return iso ? ws_launch_k<N, WS_OP, true>(L, s) : ws_launch_k<N, WS_OP, false>(L, s);
    return iso ? ws_launch_k<N, WS_CG, true>(L, s) : ws_launch_k<N, WS_CG, false>(L, s);
}

}  // namespace

bool ws_supported(int degree) { return degree >= 1 && degree <= 4; }

cudaError_t prepare_ws(int degree)
{
    switch (degree) {
    case 1: return ws_prepare_n<1>();
    case 2: return ws_prepare_n<2>();
    case 3: return ws_prepare_n<3>();
    case 4: return ws_prepare_n<4>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ws(const TmaLaunch& L, cudaStream_t s)
{
    if ((L.mode != TMODE_OP && L.mode != TMODE_CG) || L.mask) return cudaErrorInvalidValue;
    switch (L.degree) {
    case 1: return ws_launch_n<1>(L, s);
    case 2: return ws_launch_n<2>(L, s);
    case 3: return ws_launch_n<3>(L, s);
    case 4: return ws_launch_n<4>(L, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsk

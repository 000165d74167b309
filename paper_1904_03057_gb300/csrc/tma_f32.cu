// FP32 instantiation of the TMA operator / single-pass CG kernels (degrees 1..5).
#include <cstring>
#define BSK_T float
#define BSK_TMA_HIGH_DEGREE 1
#include "tma_impl.cuh"

// ---- batched single-pass CG iteration (FP32 only) ----
namespace bsk {

namespace {

template <int N>
TmaInfo& batch_info()
{
    static TmaInfo info;
    return info;
}

template <int N>
cudaError_t prepare_batch()
{
    TmaInfo& info = batch_info<N>();
    if (info.ready) return cudaSuccess;
    using LY = TLayout<float, N, TMODE_CG>;
    cudaError_t e = cudaFuncSetAttribute(k_op_tma<float, N, TMODE_CG, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::total);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_op_tma<float, N, TMODE_CG, true>, kTNT,
                                                      LY::total);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    info.grid = per_sm * sms;
    info.ready = true;
    return cudaSuccess;
}

template <int N>
cudaError_t launch_batch_n(const TmaBatchLaunch& L, cudaStream_t s)
{
    cudaError_t e = prepare_batch<N>();
    if (e != cudaSuccess) return e;
    using LY = TLayout<float, N, TMODE_CG>;
    TmaArgs<float> a;
    memset(&a, 0, sizeof a);
    a.nitems = L.nitems;
    a.work = L.work;
    a.sc = L.status;
    a.fin = FIN_CG1;
    a.batch = L.desc;
    a.nprobs = L.nprobs;
    a.parity = L.parity;
    const int grid = L.nitems < batch_info<N>().grid ? L.nitems : batch_info<N>().grid;
    if (grid < 1) return cudaSuccess;
    k_op_tma<float, N, TMODE_CG, true><<<grid, kTNT, LY::total, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t batch_problem_bytes() { return sizeof(BatchProblem<float>); }

int batch_grid(int degree)
{
    switch (degree) {
    case 1: return prepare_batch<1>() == cudaSuccess ? batch_info<1>().grid : 0;
    case 2: return prepare_batch<2>() == cudaSuccess ? batch_info<2>().grid : 0;
    case 3: return prepare_batch<3>() == cudaSuccess ? batch_info<3>().grid : 0;
    case 4: return prepare_batch<4>() == cudaSuccess ? batch_info<4>().grid : 0;
    case 5: return prepare_batch<5>() == cudaSuccess ? batch_info<5>().grid : 0;
    default: return 0;
    }
}

cudaError_t fill_batch_problem(void* host_desc, int degree, int nx, int ny, int nz, int pitch, int nzc,
                               int item0, const double (*M)[kMaxTaps], const double (*Kdt)[kMaxTaps],
                               float* const r[2], float* const q[2], float* const p[2], float* x,
                               Scalars* sc, double* partials, unsigned int* items_done, int timing,
                               int* nitems_out)
{
    BatchProblem<float>& P = *static_cast<BatchProblem<float>*>(host_desc);
    memset(&P, 0, sizeof P);
    int bx = 0, by = 0;
    switch (degree) {
    case 1: case 2: case 3: case 4: bx = TGeo<float, 4>::BX; break;
    default: bx = TGeo<float, 5>::BX; break;
    }
    by = kTY + 2 * degree;
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    auto enc = [&](CUtensorMap* m, const float* base, int bxx, int byy) -> cudaError_t {
        const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
        const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * ny * 4};
        const cuuint32_t box[3] = {(cuuint32_t)bxx, (cuuint32_t)byy, 1u};
        const cuuint32_t estr[3] = {1u, 1u, 1u};
        CUresult rr = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        return rr == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
    };
    cudaError_t e;
    for (int par = 0; par < 2; par++) {
        const float* src[3] = {r[par], q[par], p[par]};
        for (int i = 0; i < 3; i++)
            if ((e = enc(&P.tin[par][i], src[i], bx, by)) != cudaSuccess) return e;
        P.out0[par] = q[1 - par];
        P.out1[par] = r[1 - par];
        P.out2[par] = p[1 - par];
    }
    if ((e = enc(&P.tint, x, TGeo<float, 1>::IP, kTY)) != cudaSuccess) return e;
    P.xvec = x;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.pitch = pitch;
    P.tiles_x = (nx + kTX - 1) / kTX;
    P.tiles_y = (ny + kTY - 1) / kTY;
    if (nzc < 1) nzc = 1;
    if (nzc > nz) nzc = nz;
    P.tz = (nz + nzc - 1) / nzc;
    P.nitems = P.tiles_x * P.tiles_y * ((nz + P.tz - 1) / P.tz);
    P.item0 = item0;
    for (int d = 0; d < 3; d++)
        for (int j = 0; j < kMaxTaps; j++) {
            P.M[d][j] = (float)M[d][j];
            P.K[d][j] = (float)Kdt[d][j];
        }
    P.sc = sc;
    P.partials = partials;
    P.items_done = items_done;
    P.timing = timing;
    *nitems_out = P.nitems;
    return cudaSuccess;
}

cudaError_t launch_tma_batch(const TmaBatchLaunch& L, cudaStream_t s)
{
    switch (L.degree) {
    case 1: return launch_batch_n<1>(L, s);
    case 2: return launch_batch_n<2>(L, s);
    case 3: return launch_batch_n<3>(L, s);
    case 4: return launch_batch_n<4>(L, s);
    case 5: return launch_batch_n<5>(L, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsk

namespace bsk {

namespace {

// One warp per (tile, plane): OR of the mask over the tile's 64 x 24 nodes (fewer at the far
// faces), read byte by byte (rows need not start on any wider boundary).
__global__ void k_tile_occupancy(const uint8_t* __restrict__ mask, int nx, int ny, int nz, int tiles_x,
                                 int tiles_y, uint8_t* __restrict__ occ)
{
    const int lane = threadIdx.x & 31;
    const long long w = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const long long ntiles = (long long)tiles_x * tiles_y;
    if (w >= ntiles * nz) return;   // whole warps: w is uniform across the warp
    const int z = (int)(w / ntiles), tile = (int)(w % ntiles);
    const int x0 = (tile % tiles_x) * kTX, y0 = (tile / tiles_x) * kTY;
    const int cols = min(x0 + kTX, nx) - x0;
    const int rows = min(y0 + kTY, ny) - y0;
    bool any = false;
    for (int i = lane; i < rows * kTX; i += 32) {
        const int r = i / kTX, c = i % kTX;
        if (c < cols) any |= mask[((size_t)z * ny + y0 + r) * nx + x0 + c] != 0;
    }
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) occ[(size_t)z * ntiles + tile] = any ? 1 : 0;
}

}  // namespace

int tma_tiles(int nx, int ny) { return ((nx + kTX - 1) / kTX) * ((ny + kTY - 1) / kTY); }

cudaError_t launch_tile_occupancy(const uint8_t* mask, int nx, int ny, int nz, uint8_t* occ, cudaStream_t s)
{
    const int tiles_x = (nx + kTX - 1) / kTX, tiles_y = (ny + kTY - 1) / kTY;
    const long long warps = (long long)tiles_x * tiles_y * nz;
    const long long blocks = (warps + 7) / 8;
    k_tile_occupancy<<<(unsigned)blocks, 256, 0, s>>>(mask, nx, ny, nz, tiles_x, tiles_y, occ);
    return cudaGetLastError();
}

}  // namespace bsk

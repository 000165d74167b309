// tma_batch.cu -- the batched single-pass FP32 CG iteration (BATCH instantiations of op_tma.cuh),
// in three tile shapes: 64 columns x 16, 24 or 32 rows (2, 3 or 4 output rows per warp). A
// taller tile re-reads fewer y-halo rows per output (2n / (8 R) of a box) but holds more
// accumulators per thread and leaves fewer items to balance over the SMs; which one is fastest
// depends on the boxes and the degree, so the batch autotuner times them.
#include <cstring>

#include <cudaTypedefs.h>

#include "bsk_launch.h"
#include "op_tma.cuh"

namespace bsk {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 batch_encode_fn() { return tensor_map_encoder(); }

struct BatchInfo {
    bool ready = false;
    int grid = 0;   // resident blocks on the whole GPU
};

template <int N, int R>
BatchInfo& batch_info()
{
    static BatchInfo info;
    return info;
}

template <int N, int R>
cudaError_t prepare_batch()
{
    BatchInfo& info = batch_info<N, R>();
    if (info.ready) return cudaSuccess;
    using LY = TLayout<float, N, TMODE_CG, R>;
    auto kern = k_op_tma<float, N, TMODE_CG, true, R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::total);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTNT, LY::total);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    info.grid = per_sm * sms;
    info.ready = true;
    return cudaSuccess;
}

template <int N, int R>
cudaError_t launch_batch_nr(const TmaBatchLaunch& L, cudaStream_t s)
{
    cudaError_t e = prepare_batch<N, R>();
    if (e != cudaSuccess) return e;
    using LY = TLayout<float, N, TMODE_CG, R>;
    TmaArgs<float> a;
    memset(&a, 0, sizeof a);
    a.nitems = L.nitems;
    a.work = L.work;
    a.sc = L.status;
    a.fin = FIN_CG1;
    a.batch = L.desc;
    a.nprobs = L.nprobs;
    a.parity = L.parity;
    const int grid = L.nitems < batch_info<N, R>().grid ? L.nitems : batch_info<N, R>().grid;
    if (grid < 1) return cudaSuccess;
    k_op_tma<float, N, TMODE_CG, true, R><<<grid, kTNT, LY::total, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_batch_n(const TmaBatchLaunch& L, cudaStream_t s)
{
    switch (L.rows) {
    case 2: return launch_batch_nr<N, 2>(L, s);
    case 3: return launch_batch_nr<N, 3>(L, s);
    case 4:
        if constexpr (N <= kBatchMaxDegreeR4) return launch_batch_nr<N, 4>(L, s);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int N>
int batch_grid_n(int rows)
{
    switch (rows) {
    case 2: return prepare_batch<N, 2>() == cudaSuccess ? batch_info<N, 2>().grid : 0;
    case 3: return prepare_batch<N, 3>() == cudaSuccess ? batch_info<N, 3>().grid : 0;
    case 4:
        if constexpr (N <= kBatchMaxDegreeR4) return prepare_batch<N, 4>() == cudaSuccess ? batch_info<N, 4>().grid : 0;
        return 0;
    default: return 0;
    }
}

}  // namespace

size_t batch_problem_bytes() { return sizeof(BatchProblem<float>); }

bool batch_rows_supported(int degree, int rows)
{
    return degree >= 1 && degree <= 5 && (rows == 2 || rows == 3 || (rows == 4 && degree <= kBatchMaxDegreeR4));
}

int batch_grid(int degree, int rows)
{
    switch (degree) {
    case 1: return batch_grid_n<1>(rows);
    case 2: return batch_grid_n<2>(rows);
    case 3: return batch_grid_n<3>(rows);
    case 4: return batch_grid_n<4>(rows);
    case 5: return batch_grid_n<5>(rows);
    default: return 0;
    }
}

cudaError_t fill_batch_problem(void* host_desc, int degree, int rows, int nx, int ny, int nz, int pitch, int nzc,
                               int item0, const double (*M)[kMaxTaps], const double (*Kdt)[kMaxTaps],
                               float* const r[2], float* const q[2], float* const p[2], float* x,
                               Scalars* sc, double* partials, unsigned int* items_done, int timing,
                               int* nitems_out)
{
    if (!batch_rows_supported(degree, rows)) return cudaErrorInvalidValue;
    BatchProblem<float>& P = *static_cast<BatchProblem<float>*>(host_desc);
    memset(&P, 0, sizeof P);
    const int ty = 8 * rows;
    const int bx = degree <= 4 ? TGeo<float, 4>::BX : TGeo<float, 5>::BX;   // BX depends on the degree only
    const int by = ty + 2 * degree;
    auto fn = batch_encode_fn();
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
    if ((e = enc(&P.tint, x, TGeo<float, 1>::IP, ty)) != cudaSuccess) return e;
    P.xvec = x;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.pitch = pitch;
    P.tiles_x = (nx + kTX - 1) / kTX;
    P.tiles_y = (ny + ty - 1) / ty;
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

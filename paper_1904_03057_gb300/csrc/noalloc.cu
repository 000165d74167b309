// noalloc.cu -- residual_noalloc: r = b - A x with r.r and b.b, for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another component owns the device
// memory budget (a host application that hands this library pre-allocated buffers and forbids
// allocation inside its solver callbacks), or code that must not allocate between two points
// where allocation would synchronise the device. Everything else in this library allocates its
// work space in bsk_create. This entry point needs no handle: its only scratch (the FP64 CG-style
// scalar block and the per-block partial sums of its two reductions) lives in one file-scope
// __device__ array that every GPU loading the library holds until the process exits.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "bsk.h"
#include "bsk_launch.h"

namespace {

// Largest operator grid (blocks of the general operator kernel) the static scratch can reduce.
// The general kernel's grid has ceil(nx/32) * ceil(ny/16) blocks per z-slab and a single slab
// once that product reaches 1216, so the bound is ceil(nx/32) * ceil(ny/16) <= 16384 (about
// 8.4 M nodes per x-y plane), whatever nz is.
constexpr size_t kNoAllocMaxBlocks = 16384;

struct NoAllocScratch {
    bsk::Scalars sc;
    double partials[2 * kNoAllocMaxBlocks];
};

__device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
void* g_noalloc_addr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device
bool g_noalloc_prepared[kMaxDevices][2][6] = {};   // kernel set-up done: device, FP64?, degree

int noalloc_fail(int code, const char* msg) { return bsk::set_error(code, msg); }

// Host code cannot use g_noalloc_scratch as a device address (on the host that name is only a
// stand-in), so each device's address is fetched once, with that device current. The operator
// kernels' shared-memory limits are set once per device, precision and degree at the same time.
int scratch_address(void** out, bool fp64, int degree)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(BSK_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(BSK_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return noalloc_fail(BSK_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        g_noalloc_addr[dev] = p;
    }
    if (!g_noalloc_prepared[dev][fp64][degree]) {
        const cudaError_t e = fp64 ? bsk::prepare_op<double>(degree) : bsk::prepare_op<float>(degree);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return noalloc_fail(BSK_ECUDA, "kernel set-up failed");
        }
        g_noalloc_prepared[dev][fp64][degree] = true;
    }
    *out = g_noalloc_addr[dev];
    return BSK_OK;
}

}  // namespace

extern "C" int residual_noalloc(const bsk_problem* prob, int precision, const void* x, const void* b,
                                void* r, double* rr, double* bb, void* stream)
{
    if (!prob || !x || !b || !r || !rr || !bb) return noalloc_fail(BSK_EINVAL, "null argument");
    const int n = prob->degree;
    if (n < 1 || n > 5) return noalloc_fail(BSK_EINVAL, "degree outside 1..5");
    if (prob->nx < n || prob->ny < n || prob->nz < n)
        return noalloc_fail(BSK_EINVAL, "each axis needs at least degree unknowns");
    if (!(prob->hx > 0) || !(prob->hy > 0) || !(prob->hz > 0) || !(prob->dt >= 0))
        return noalloc_fail(BSK_EINVAL, "grid steps must be > 0 and dt >= 0");
    if (precision != BSK_F64 && precision != BSK_F32)
        return noalloc_fail(BSK_EINVAL, "precision must be BSK_F64 or BSK_F32");
    const size_t blocks = bsk::op_grid_blocks(prob->nx, prob->ny, prob->nz, n);
    if (blocks > kNoAllocMaxBlocks) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "grid too large for the static scratch: %zu operator blocks, at most %zu "
                 "(ceil(nx/32) * ceil(ny/16) <= 16384, about 8.4 M nodes per x-y plane, any nz)",
                 blocks, kNoAllocMaxBlocks);
        return noalloc_fail(BSK_EINVAL, msg);
    }
    const size_t es = precision == BSK_F64 ? sizeof(double) : sizeof(float);
    const size_t len = (size_t)prob->nx * prob->ny * prob->nz;
    const char *px = (const char*)x, *pb = (const char*)b, *pr = (const char*)r;
    if ((pr < px + len * es && px < pr + len * es) || (pr < pb + len * es && pb < pr + len * es))
        return noalloc_fail(BSK_EINVAL, "r overlaps x or b");

    cudaStream_t st = (cudaStream_t)stream;
    // every call reads its result back and synchronises the stream, which a capture cannot hold
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(BSK_ECUDA, "cudaStreamIsCapturing failed");
    }
    if (cap != cudaStreamCaptureStatusNone)
        return noalloc_fail(BSK_EINVAL, "residual_noalloc cannot run while its stream is capturing");

    void* base = nullptr;
    if (int rc = scratch_address(&base, es == sizeof(double), n)) return rc;
    NoAllocScratch* s = static_cast<NoAllocScratch*>(base);
    // the scratch keeps the previous call's contents: the reduction counter must start at zero
    cudaError_t e = cudaMemsetAsync(&s->sc, 0, sizeof(bsk::Scalars), st);
    if (e != cudaSuccess) return noalloc_fail(BSK_ECUDA, "cudaMemsetAsync failed");

    bsk::OpLaunch L;
    memset(&L, 0, sizeof L);
    L.mode = bsk::MODE_RES;
    L.degree = n;
    L.nx = prob->nx;
    L.ny = prob->ny;
    L.nz = prob->nz;
    L.mask = prob->mask;
    const double hs[3] = {prob->hx, prob->hy, prob->hz};
    for (int d = 0; d < 3; d++) {
        double m[bsk::kMaxTaps] = {0}, k[bsk::kMaxTaps] = {0};
        bspline_kernels(n, hs[d], m, k);
        for (int j = 0; j < 2 * n + 1; j++) {
            L.M[d][j] = m[j];
            L.Kdt[d][j] = prob->dt * k[j];
        }
    }
    L.in0 = x;
    L.b = b;
    L.out0 = r;
    L.sc = &s->sc;
    L.partials = s->partials;
    L.fin = bsk::FIN_RES_TRUE;
    e = es == sizeof(double) ? bsk::launch_op<double>(L, st) : bsk::launch_op<float>(L, st);
    if (e != cudaSuccess) return noalloc_fail(BSK_ECUDA, "operator launch failed");
    bsk::Scalars out;
    e = cudaMemcpyAsync(&out, &s->sc, sizeof out, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(BSK_ECUDA, "result copy failed");
    *rr = out.rr_true;
    *bb = out.bb_true;
    return BSK_OK;
}

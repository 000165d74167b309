// op_tma.cuh -- the fast operator / CG kernel for unmasked box problems whose rows are 16-byte
// multiples (TMA-addressable): A x, b - A x, and one whole CG iteration in a single pass.
//
// Structure (arXiv:1904.03057 section 2.4: A = Mz My Mx + dt (Kz My Mx + Mz Ky Mx + Mz My Kx)
// applied as separable shift-invariant band convolutions, Fig. FiltAlg). The three sweeps are
// reordered so that no sweep is recomputed on a z halo:
//     A x = (Mz + dt Kz) U + Mz V,    U = My Mx x,    V = dt (Ky Mx + My Kx) x.
// A block owns a 64 x 24 (x, y) tile and marches along z. Per input plane:
//   1. TMA brings the tile plus its halo (n rows, 4 or 8 columns) of every input vector into a
//      shared-memory stage (double/triple buffered, mbarrier completion, no multicast); box faces
//      are completed by odd reflection in shared memory, reflected planes by a sign.
//   2. x-sweep in shared memory: MX = Mx x, KX = dt Kx x on the 64-column tile x (24+2n) rows.
//   3. y-sweep, in registers of the thread that owns the column pair: U = My MX,
//      V = dt Ky MX + My KX (packed f32x2 arithmetic for FP32).
//   4. z-sweep as a push: the plane's U, V are added, with the 2n+1 z taps, into a ring of 2n+1
//      per-thread accumulators of the output planes z-n .. z+n; output plane z-n is complete and
//      leaves the kernel straight from registers.
// A node mask (principal submatrix of the box operator) needs no staging: every input the
// kernel reads is zero on inactive nodes already (the solvers keep their vectors masked), so
// only the operator outputs are multiplied by the mask, read as two bits per output pair from a
// bit-packed copy (1/8 byte per unknown).
// Blocks are persistent and walk a static list of (tile, z-chunk) items. In CG mode the staged
// value is the new search direction p_m = (r - alpha q) + beta p of the previous iteration's
// vectors, and the pass also writes r_m, p_m, x_m = x + alpha p and reduces r.r, p.Ap, Ap.Ap
// (single-synchronisation CG, see finalize_cg1).
#pragma once

#include <type_traits>

#include "bsk_device.cuh"
#include "dfloat.cuh"
#include "tma_util.cuh"

namespace bsk {

constexpr int kTX = 64;     // output columns per tile
constexpr int kTR = 3;      // output rows per warp of the single-problem kernels
constexpr int kTY = 8 * kTR;   // their output rows per tile (8 warps x 3 rows)
constexpr int kTNT = 256;   // threads per block

template <typename T>
struct TmaArgs {
    CUtensorMap tin[3];   // halo boxes: OP/RES {x}; CG {p_{m-1}, q_{m-1}, p_{m-2}} (batched CG:
                          // {r, q, p} of the previous iteration)
    CUtensorMap tint;     // interior box: RES {b}; CG {x}
    T* out0;              // OP y; RES r; CG q_m = A p_m
    T* out1;              // batched CG r_m (single-problem CG keeps no r)
    T* out2;              // CG p_m
    T* xvec;              // CG x, updated in place
    const uint32_t* mbits;   // bit-packed node mask or null: row (z, y) holds mwords 32-bit words,
                             // bit i of word w = node x = 32 w + i; outputs (q, r) are zeroed
                             // where it is 0 and the inputs must already be zero there
                             // (principal submatrix)
    int mwords;
    const uint8_t* occ;   // with a mask: occ[z * tiles + tile] != 0 iff tile has an active node in
                          // plane z; items with none are skipped (their outputs stay zero)
    int nx, ny, nz;
    // OP on a z-slab: the nz local planes are planes z_off .. of a grid of nz_glob planes, and
    // tin[0] holds nz + 2 zpad planes (plane i = global plane z_off - zpad + i); odd reflection
    // at the global faces only. A whole grid: z_off = 0, nz_glob = nz, zpad = 0.
    int z_off, nz_glob, zpad;
    int pitch;            // elements per row in memory (>= nx; rows of 16-byte multiples)
    int tiles_x, tiles_y, tz, nitems;
    T M[3][kMaxTaps];     // per-axis mass kernels, index j + n
    T K[3][kMaxTaps];     // per-axis stiffness kernels times dt
    Scalars* sc;
    double* partials;
    unsigned int* work;   // [0] next item, [1] blocks finished; both zero between launches
    int fin;
    // batched CG (BATCH kernels): the problems, their first items, and the ping-pong parity
    const void* batch;    // BatchProblem<T>[nprobs] in device memory
    int nprobs;
    int parity;
};

// One problem of a batched CG pass, in device memory. The pass with parity P reads the halo
// boxes tin[P] = (r, q, p) and writes (q, r, p) to out*[P]; x is updated in place.
template <typename T>
struct BatchProblem {
    CUtensorMap tin[2][3];
    CUtensorMap tint;            // interior box of x
    T* out0[2];                  // q
    T* out1[2];                  // r
    T* out2[2];                  // p
    T* xvec;
    int nx, ny, nz, pitch;
    int tiles_x, tiles_y, tz, nitems, item0;   // item0: first item of this problem in the pass
    T M[3][kMaxTaps];
    T K[3][kMaxTaps];
    Scalars* sc;
    double* partials;            // 3 doubles per item of this problem
    unsigned int* items_done;    // items of this problem finished in the current pass
    int timing;                  // non-zero: skip the finaliser (kernel timing passes)
    int pad[5];
};

// Tile geometry: 64 columns x 8 R rows (R output rows per warp; the batched kernels come in
// R = 2, 3, 4, the single-problem kernels use R = 3).
template <typename T, int N, int R = kTR>
struct TGeo {
    static constexpr int L = 2 * N + 1;
    static constexpr int TY = 8 * R;                    // output rows per tile
    static constexpr int HL = N <= 4 ? 4 : 8;          // halo columns staged on each side
    static constexpr int BX = kTX + 2 * HL + 4;         // box width; +4 columns spread smem banks
    static constexpr int HY = TY + 2 * N;               // box height (tile rows + y halo)
    static constexpr int MXP = kTX + 4;                 // row pitch of the x-sweep results
    // interior box (b or x) width = row pitch of it and of the ring: 16 bytes over the tile,
    // so that threads on consecutive rows hit distinct shared-memory banks
    static constexpr int IP = kTX + 16 / (int)sizeof(T);
    static constexpr int WIN = 8 + 2 * HL;              // x-window loaded per 8 outputs
};

template <typename T, int N, int MODE, int R = kTR>
struct TLayout {
    using G = TGeo<T, N, R>;
    static constexpr int NIN = MODE == TMODE_CG ? 3 : 1;
    static constexpr int NINT = MODE == TMODE_OP ? 0 : 1;
    static constexpr size_t rnd(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t in_bytes = rnd(sizeof(T) * G::HY * G::BX);
    static constexpr size_t int_bytes = rnd(sizeof(T) * G::TY * G::IP);
    static constexpr size_t stage_bytes = NIN * in_bytes + NINT * int_bytes;
    static constexpr int S = MODE == TMODE_OP ? 4 : 2;   // pipeline stages
    static constexpr size_t off_mx = S * stage_bytes;
    static constexpr size_t mx_bytes = rnd(sizeof(T) * G::HY * G::MXP);
    static constexpr size_t off_ring = off_mx + 2 * mx_bytes;
    static constexpr size_t ring_bytes = MODE == TMODE_OP ? 0 : (N + 1) * int_bytes;
    static constexpr size_t off_bar = off_ring + ring_bytes;
    static constexpr size_t total = off_bar + 64;
    static constexpr uint32_t tx_bytes =
        (uint32_t)(NIN * sizeof(T) * G::HY * G::BX + NINT * sizeof(T) * G::TY * G::IP);
};

// Packed pair arithmetic: f32x2 instructions for FP32, two scalar operations for FP64.
template <typename T> struct P2;
template <> struct P2<float> {
    using t = float2;
    static __device__ __forceinline__ t mk(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ t fma(t a, t b, t c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ t add(t a, t b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ t zero() { return make_float2(0.f, 0.f); }
};
template <> struct P2<double> {
    using t = double2;
    static __device__ __forceinline__ t mk(double a) { return make_double2(a, a); }
    static __device__ __forceinline__ t fma(t a, t b, t c)
    {
        return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
    }
    static __device__ __forceinline__ t add(t a, t b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ t zero() { return make_double2(0.0, 0.0); }
};

// Double-float pairs (the FP64-accurate residual on the FP32 pipes, T = dfl): boxes arrive as
// FP64 and are split in shared memory; every tap is an exact product plus a two-sum.
template <> struct P2<dfl> {
    using t = dfl2;
    static __device__ __forceinline__ t mk(dfl a) { return dfl2{a, a}; }
    static __device__ __forceinline__ t fma(t a, t b, t c) { return dfl2{df_fma(a.x, b.x, c.x), df_fma(a.y, b.y, c.y)}; }
    static __device__ __forceinline__ t add(t a, t b) { return dfl2{df_add(a.x, b.x), df_add(a.y, b.y)}; }
    static __device__ __forceinline__ t zero() { return dfl2{dfl(0.f, 0.f), dfl(0.f, 0.f)}; }
};
__device__ __forceinline__ dfl operator+(dfl a, dfl b) { return df_add(a, b); }

// Compensated (Kahan) running sum in the element precision; converted to FP64 once per block.
template <typename T>
struct KSum {
    T s = T(0), c = T(0);
    __device__ __forceinline__ void add(T v)
    {
        const T y = v - c;
        const T t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// W consecutive elements from 16-byte aligned shared memory, in 16-byte vector loads.
template <typename T, int W>
__device__ __forceinline__ void load_window(T (&v)[W], const T* src)
{
    static_assert(W % 4 == 0, "whole vectors");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < W / 4; q++) {
            const float4 f = reinterpret_cast<const float4*>(src)[q];
            v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
        }
    } else {
        struct alignas(16) Pair { T a, b; };
#pragma unroll
        for (int q = 0; q < W / 2; q++) {
            const Pair f = reinterpret_cast<const Pair*>(src)[q];
            v[2 * q] = f.a; v[2 * q + 1] = f.b;
        }
    }
}

// Odd reflection of the ghost rows / columns of one staged box that the sweeps read (at most n
// on each side); ghosts further out stay as loaded (zero) and feed no output that is stored.
template <typename T, int N, int R = kTR>
__device__ __forceinline__ void patch_rows(T* box, int y0, int ny)
{
    using G = TGeo<T, N, R>;
    // box row br <-> grid row y0 - N + br; ghosts read: [0, N) when y0 == 0, and
    // [ny - y0 + N, ny - y0 + 2N) at the far face
    const int lo_n = (y0 == 0) ? N : 0;
    const int hi_b = ny - y0 + N;
    const int hi_n = (hi_b < G::HY) ? min(N, G::HY - hi_b) : 0;
    const int cnt = (lo_n + hi_n) * G::BX;
    for (int i = threadIdx.x; i < cnt; i += kTNT) {
        const int rr = i / G::BX, bc = i - rr * G::BX;
        const int br = rr < lo_n ? rr : hi_b + (rr - lo_n);
        const int gy = y0 - N + br;
        int src = 0;
        const int s = reflect_index(gy, ny, src);
        const int sr = src - (y0 - N);
        box[br * G::BX + bc] = (s && sr >= 0 && sr < G::HY) ? (T)s * box[sr * G::BX + bc] : T(0);
    }
}

template <typename T, int N, int R = kTR>
__device__ __forceinline__ void patch_cols(T* box, int x0, int nx)
{
    using G = TGeo<T, N, R>;
    // box column bc <-> grid column x0 - HL + bc; ghosts read: [HL - N, HL) when x0 == 0, and
    // [nx - x0 + HL, nx - x0 + HL + N) at the far face
    const int lo_n = (x0 == 0) ? N : 0;
    const int hi_b = nx - x0 + G::HL;
    const int hi_n = (hi_b < G::BX) ? min(N, G::BX - hi_b) : 0;
    const int cnt = (lo_n + hi_n) * G::HY;
    for (int i = threadIdx.x; i < cnt; i += kTNT) {
        const int cc = i / G::HY, br = i - cc * G::HY;
        const int bc = cc < lo_n ? (G::HL - N + cc) : hi_b + (cc - lo_n);
        const int gx = x0 - G::HL + bc;
        int src = 0;
        const int s = reflect_index(gx, nx, src);
        const int sc = src - (x0 - G::HL);
        box[br * G::BX + bc] = (s && sc >= 0 && sc < G::BX) ? (T)s * box[br * G::BX + sc] : T(0);
    }
}

// z push of one plane into the accumulator ring (slot of output plane z + d is (J + d) mod L),
// then hand back the completed output plane z - n (slot (J - n) mod L) and clear its slot.
template <typename T2, typename PP, int N, int R, int J>
__device__ __forceinline__ void push_plane(T2 (&acc)[R][2 * N + 1], const T2 (&U)[R], const T2 (&V)[R],
                                           const T2 (&w1z)[N + 1], const T2 (&mz)[N + 1], T2 (&q)[R])
{
    constexpr int L = 2 * N + 1;
#pragma unroll
    for (int t = 0; t < R; t++) {
#pragma unroll
        for (int dd = -N; dd <= N; dd++) {
            const int sl = ((J + dd) % L + L) % L;
            const int ad = dd < 0 ? -dd : dd;
            acc[t][sl] = PP::fma(w1z[ad], U[t], acc[t][sl]);
            acc[t][sl] = PP::fma(mz[ad], V[t], acc[t][sl]);
        }
        constexpr int fs = ((J - N) % L + L) % L;
        q[t] = acc[t][fs];
        acc[t][fs] = PP::zero();
    }
}

template <typename T2, typename PP, int N, int R>
__device__ __forceinline__ void push_dispatch(int j, T2 (&acc)[R][2 * N + 1], const T2 (&U)[R],
                                              const T2 (&V)[R], const T2 (&w1z)[N + 1],
                                              const T2 (&mz)[N + 1], T2 (&q)[R])
{
    switch (j) {
    case 0: push_plane<T2, PP, N, R, 0>(acc, U, V, w1z, mz, q); break;
    case 1: push_plane<T2, PP, N, R, 1>(acc, U, V, w1z, mz, q); break;
    case 2: push_plane<T2, PP, N, R, 2>(acc, U, V, w1z, mz, q); break;
    default:
        if constexpr (N >= 2) {
            switch (j) {
            case 3: push_plane<T2, PP, N, R, 3>(acc, U, V, w1z, mz, q); break;
            case 4: push_plane<T2, PP, N, R, 4>(acc, U, V, w1z, mz, q); break;
            default:
                if constexpr (N >= 3) {
                    switch (j) {
                    case 5: push_plane<T2, PP, N, R, 5>(acc, U, V, w1z, mz, q); break;
                    case 6: push_plane<T2, PP, N, R, 6>(acc, U, V, w1z, mz, q); break;
                    default:
                        if constexpr (N >= 4) {
                            switch (j) {
                            case 7: push_plane<T2, PP, N, R, 7>(acc, U, V, w1z, mz, q); break;
                            case 8: push_plane<T2, PP, N, R, 8>(acc, U, V, w1z, mz, q); break;
                            default:
                                if constexpr (N >= 5) {
                                    if (j == 9) push_plane<T2, PP, N, R, 9>(acc, U, V, w1z, mz, q);
                                    else push_plane<T2, PP, N, R, 10>(acc, U, V, w1z, mz, q);
                                }
                            }
                        }
                    }
                }
            }
        }
    }
}

template <typename T, int N, int MODE, bool BATCH, int R = kTR>
__global__ void __launch_bounds__(kTNT, (sizeof(T) == 4 && N <= 4 && !BATCH) ? 2 : 1)
    k_op_tma(const __grid_constant__ TmaArgs<T> a)
{
    using G = TGeo<T, N, R>;
    using LY = TLayout<T, N, MODE, R>;
    constexpr int TY = G::TY;
    static_assert(BATCH || R == kTR, "single-problem kernels use 64 x 24 tiles");
    using PP = P2<T>;
    using T2 = typename PP::t;
    constexpr int L = G::L, HY = G::HY, BX = G::BX, MXP = G::MXP, HL = G::HL, WIN = G::WIN, IP = G::IP;
    constexpr int S = LY::S;
    constexpr int NIN = LY::NIN;
    static_assert(LY::total <= 227 * 1024, "shared memory budget");
    static_assert(WIN % 4 == 0 && HL % 2 == 0, "window loads are 16-byte vectors, pairs aligned");
    static_assert(!BATCH || MODE == TMODE_CG, "batched passes are CG iterations");

    extern __shared__ __align__(128) unsigned char smem[];
    T* MXs = reinterpret_cast<T*>(smem + LY::off_mx);
    T* KXs = reinterpret_cast<T*>(smem + LY::off_mx + LY::mx_bytes);
    T* ring = reinterpret_cast<T*>(smem + LY::off_ring);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + LY::off_bar);
    __shared__ int s_abort, s_item, s_prob, s_last;
    __shared__ uint32_t s_issued, s_wait_from;   // loads issued / first load not yet consumed
    __shared__ double s_red[3 * (kTNT / 32)];
    const BatchProblem<T>* probs = static_cast<const BatchProblem<T>*>(a.batch);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (!BATCH && MODE == TMODE_CG) {
        if (*(volatile int*)&a.sc->done) return;   // uniform over the grid
    }
    // item fetch (thread 0): next item of the queue and, for a batch, its problem
    auto fetch = [&]() {
        const int it = (int)atomicAdd(&a.work[0], 1u);
        s_item = it;
        if (BATCH && it < a.nitems) {
            int lo = 0, hi = a.nprobs - 1;   // last problem with item0 <= it
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (probs[mid].item0 <= it) lo = mid; else hi = mid - 1;
            }
            s_prob = lo;
        }
    };
    if (tid == 0) {
        for (int s = 0; s < S; s++) mbar_init(&bars[s], 1);
        fence_mbar_init();
        if (!BATCH) {
            for (int i = 0; i < NIN; i++) prefetch_tensormap(&a.tin[i]);
            if (LY::NINT) prefetch_tensormap(&a.tint);
        }
        s_abort = 0;
        s_issued = 0;
        s_wait_from = 0;
        s_prob = 0;
        fetch();
    }
    __syncthreads();

    // ---- the current problem (fixed for a single problem, per item for a batch) ----
    const CUtensorMap *tin0 = &a.tin[0], *tin1 = &a.tin[1], *tin2 = &a.tin[2], *tint = &a.tint;
    T *out0 = a.out0, *out1 = a.out1, *out2 = a.out2, *xvec = a.xvec;
    int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    int tiles_x = a.tiles_x, tiles_y = a.tiles_y, tz = a.tz, item0 = 0;
    Scalars* sc = a.sc;
    constexpr bool DF = std::is_same<T, dfl>::value;   // double-float passes (FP64 vectors)
    static_assert(!DF || (MODE != TMODE_CG && !BATCH), "double-float: operator and residual passes only");
    // Single-problem CG passes keep no r: pass m reads p_{m-1}, p_{m-2} and q_{m-1} and rebuilds
    // r_{m-1} = p_{m-1} - beta_{m-2} p_{m-2} (the p recurrence solved for r), which saves the r
    // write and its re-read (28 instead of 32 bytes per unknown). Batched passes keep r.
    constexpr bool RFOLD = (MODE == TMODE_CG && !BATCH);
    T alpha = T(0), beta = T(0), beta_prev = T(0);
    if constexpr (!BATCH && MODE == TMODE_CG) {
        alpha = (T)a.sc->alpha;
        beta = (T)a.sc->beta;
        beta_prev = (T)a.sc->beta_prev;
    }
    // packed taps: W1 = Mz + dt Kz and Mz for the z push; My and dt Ky for the y-sweep;
    // Mx and dt Kx for the x-sweep
    T2 w1z[N + 1], mz[N + 1], my[N + 1], ky[N + 1], mxp[N + 1], kxp[N + 1];
    auto load_taps = [&](const T (&M)[3][kMaxTaps], const T (&K)[3][kMaxTaps]) {
#pragma unroll
        for (int j = 0; j <= N; j++) {
            w1z[j] = PP::mk(M[2][N + j] + K[2][N + j]);
            mz[j] = PP::mk(M[2][N + j]);
            my[j] = PP::mk(M[1][N + j]);
            ky[j] = PP::mk(K[1][N + j]);
            mxp[j] = PP::mk(M[0][N + j]);
            kxp[j] = PP::mk(K[0][N + j]);
        }
    };
    if (!BATCH) load_taps(a.M, a.K);
    int cur_prob = -1;

    // x-sweep task of this thread (one task per thread when 8 * HY <= block size)
    constexpr int NTASK = 8 * HY;
    constexpr bool ONE_TASK = NTASK <= kTNT;
    const int xrow = tid % HY, xg = tid / HY;
    // y-sweep / z push: this thread's column pair and first row in the x-sweep results
    const T* mxb = MXs + R * warp * MXP + 2 * lane;
    const T* kxb = KXs + R * warp * MXP + 2 * lane;

    using Acc = std::conditional_t<DF, float, T>;
    KSum<Acc> d0, d1, d2;
    double s0 = 0.0, s1 = 0.0;   // DF: plain FP64 sums of r.r and b.b
    uint32_t cnt = 0;   // planes consumed by this block before the current item

    for (;;) {
        const int item_g = s_item;
        if (item_g >= a.nitems) break;
        if (BATCH) {
            const int pi = s_prob;
            const BatchProblem<T>& P = probs[pi];
            if (*(volatile int*)&P.sc->done) {   // converged earlier: its items are skipped
                __syncthreads();
                if (tid == 0) fetch();
                __syncthreads();
                continue;
            }
            if (pi != cur_prob) {
                cur_prob = pi;
                tin0 = &P.tin[a.parity][0];
                tin1 = &P.tin[a.parity][1];
                tin2 = &P.tin[a.parity][2];
                tint = &P.tint;
                out0 = P.out0[a.parity];
                out1 = P.out1[a.parity];
                out2 = P.out2[a.parity];
                xvec = P.xvec;
                nx = P.nx; ny = P.ny; nz = P.nz; pitch = P.pitch;
                tiles_x = P.tiles_x; tiles_y = P.tiles_y; tz = P.tz; item0 = P.item0;
                sc = P.sc;
                if constexpr (BATCH) {
                    alpha = (T)P.sc->alpha;
                    beta = (T)P.sc->beta;
                }
                load_taps(P.M, P.K);
            }
        }
        const int item = item_g - item0;
        const int ntiles = tiles_x * tiles_y;
        const int tile = item % ntiles, zc = item / ntiles;
        const int x0 = (tile % tiles_x) * kTX, y0 = (tile / tiles_x) * TY;
        const int z0 = zc * tz, z1 = min(z0 + tz, nz);
        const int zs = z0 - N;
        const int np = (z1 - z0) + 2 * N;
        const bool patch_x = (x0 == 0) || (x0 + kTX + N > nx);
        const bool patch_y = (y0 == 0) || (y0 + TY + N > ny);
        // z-slab geometry (single-problem OP passes; a batch problem is always a whole grid)
        const int z_off = BATCH ? 0 : a.z_off, nz_glob = BATCH ? nz : a.nz_glob, zpad = BATCH ? 0 : a.zpad;
        if (!BATCH && a.occ) {
            // brick occupancy: an item whose output box holds no active node is left out. Its
            // outputs are zero and already zero in the solvers' vectors (which are zero off the
            // mask from creation on), and it adds nothing to the dot products.
            bool act = false;
            for (int zt = z0 + tid; zt < z1; zt += kTNT) act |= a.occ[(size_t)zt * ntiles + tile] != 0;
            if (!__syncthreads_or(act)) {
                if (tid == 0) fetch();
                __syncthreads();
                continue;
            }
        }

        auto issue = [&](int k) {   // plane k of this item -> stage (cnt + k) % S
            const uint32_t c = cnt + (uint32_t)k;
            unsigned char* st = smem + (c % S) * LY::stage_bytes;
            int zsrc = 0;
            const int zz = zs + k;
            // global plane z_off + zz, reflected about the global faces, as a plane of the input
            // array (a face plane: any plane, scaled by 0)
            if (!reflect_index(z_off + zz, nz_glob, zsrc)) zsrc = z_off;
            zsrc += zpad - z_off;
            uint64_t* bar = &bars[c % S];
            mbar_arrive_expect_tx(bar, LY::tx_bytes);
            const CUtensorMap* maps[3] = {tin0, tin1, tin2};
            for (int i = 0; i < NIN; i++)
                tma_load_3d(st + i * LY::in_bytes, maps[i], bar, x0 - HL, y0 - N, zsrc);
            if (LY::NINT) {
                const int zi = min(max(zz, 0), nz - 1);
                tma_load_3d(st + NIN * LY::in_bytes, tint, bar, x0, y0, zi);
            }
            s_issued = c + 1;
        };
        if (tid == 0) {
            for (int k = 0; k < S && k < np; k++) issue(k);
        }

        T2 acc[R][L];
#pragma unroll
        for (int t = 0; t < R; t++)
#pragma unroll
            for (int s = 0; s < L; s++) acc[t][s] = PP::zero();

        int jslot = 0;   // k mod L
        for (int k = 0; k < np; k++) {
            const int z = zs + k;
            const uint32_t c = cnt + (uint32_t)k;
            unsigned char* st = smem + (c % S) * LY::stage_bytes;
            T* in0 = reinterpret_cast<T*>(st);
            T* in1 = reinterpret_cast<T*>(st + LY::in_bytes);
            T* in2 = reinterpret_cast<T*>(st + 2 * LY::in_bytes);
            T* inint = reinterpret_cast<T*>(st + NIN * LY::in_bytes);

            // every thread waits on the stage's mbarrier itself (which also makes the TMA data
            // visible to it), so no block barrier is needed here; a wait that gives up is
            // reported after the x-sweep's barrier, which every thread still reaches
            if (!mbar_wait_bounded(&bars[c % S], (c / S) & 1u, 2000000000ull)) {
                s_abort = 1;
                s_wait_from = c;
            }

            if constexpr (DF) {
                // the box holds FP64 as loaded: reflect in FP64, then split in place
                double* bd = reinterpret_cast<double*>(in0);
                if (patch_y) {
                    patch_rows<double, N, R>(bd, y0, ny);
                    __syncthreads();
                }
                if (patch_x) {
                    patch_cols<double, N, R>(bd, x0, nx);
                    __syncthreads();
                }
                for (int i = tid; i < HY * BX; i += kTNT) {
                    const double dv = bd[i];
                    in0[i] = df_from_double(dv);
                }
                __syncthreads();
            } else {
                if (patch_y) {
                    patch_rows<T, N, R>(in0, y0, ny);
                    if (NIN > 1) { patch_rows<T, N, R>(in1, y0, ny); patch_rows<T, N, R>(in2, y0, ny); }
                    __syncthreads();
                }
                if (patch_x) {
                    patch_cols<T, N, R>(in0, x0, nx);
                    if (NIN > 1) { patch_cols<T, N, R>(in1, x0, nx); patch_cols<T, N, R>(in2, x0, nx); }
                    __syncthreads();
                }
            }

            {
                int zsrc = 0;
                const int zsi = reflect_index(z_off + z, nz_glob, zsrc);   // 1, -1 (mirror plane) or 0 (face)
                const T zsgn = (T)zsi;
                const bool zint = (z >= z0 && z < z1);
                const int rslot = zint ? (z - z0) % (N + 1) : 0;
                // ---- x-sweep: task = (row, group of 8 output columns) ----
#pragma unroll 1
                for (int t = tid; t < NTASK; t += kTNT) {
                    int row, g;
                    if constexpr (ONE_TASK) { row = xrow; g = xg; }
                    else { row = t % HY; g = t / HY; }
                    T v[WIN];
                    load_window<T, WIN>(v, in0 + row * BX + 8 * g);
                    const bool interior = zint && row >= N && row < N + TY;
                    if constexpr (MODE == TMODE_CG) {
                        // p_m = (r - alpha q) + beta p of the previous iteration's vectors; with
                        // RFOLD the boxes are (p_{m-1}, q_{m-1}, p_{m-2}) and r is rebuilt first
                        T qv[WIN], pv[WIN];
                        load_window<T, WIN>(qv, in1 + row * BX + 8 * g);
                        load_window<T, WIN>(pv, in2 + row * BX + 8 * g);
                        T rc[8], pold[8];
#pragma unroll
                        for (int i = 0; i < WIN; i++) {
                            if constexpr (RFOLD) {
                                const T pc = v[i];                              // p_{m-1}
                                const T rn = fma(-alpha, qv[i], fma(-beta_prev, pv[i], pc));
                                if (i >= HL && i < HL + 8) { rc[i - HL] = rn; pold[i - HL] = pc; }
                                v[i] = fma(beta, pc, rn);
                            } else {
                                const T rn = fma(-alpha, qv[i], v[i]);
                                if (i >= HL && i < HL + 8) { rc[i - HL] = rn; pold[i - HL] = pv[i]; }
                                v[i] = fma(beta, pv[i], rn);
                            }
                        }
                        if (interior) {
                            const int gy = y0 + row - N;
                            const T* xin = inint + (row - N) * IP + 8 * g;
                            T* rg = ring + rslot * (TY * IP) + (row - N) * IP + 8 * g;
                            T xi8[8];
                            load_window<T, 8>(xi8, xin);
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                const int gx = x0 + 8 * g + 4 * h;
                                T pn4[4], rn4[4], xn4[4];
                                T part = T(0);
#pragma unroll
                                for (int e = 0; e < 4; e++) {
                                    pn4[e] = v[HL + 4 * h + e];   // interior plane: no sign
                                    rn4[e] = rc[4 * h + e];
                                    xn4[e] = fma(alpha, pold[4 * h + e], xi8[4 * h + e]);
                                    if (gx + e < nx) part = fma(rn4[e], rn4[e], part);
                                }
                                if constexpr (sizeof(T) == 4) {
                                    *reinterpret_cast<float4*>(rg + 4 * h) = make_float4(pn4[0], pn4[1], pn4[2], pn4[3]);
                                } else {
                                    *reinterpret_cast<T2*>(rg + 4 * h) = T2{pn4[0], pn4[1]};
                                    *reinterpret_cast<T2*>(rg + 4 * h + 2) = T2{pn4[2], pn4[3]};
                                }
                                if (gy < ny && gx < nx) {
                                    // rows are padded to 16-byte multiples: a partial group of
                                    // four writes into the padding, which no kernel reads. The
                                    // outputs are streamed (evict-first), so that they do not push
                                    // the halo rows neighbouring tiles still read out of L2.
                                    const size_t o = ((size_t)z * ny + gy) * pitch + gx;
                                    d0.add(part);
                                    if constexpr (sizeof(T) == 4) {
                                        if constexpr (!RFOLD)
                                            __stcs(reinterpret_cast<float4*>(out1 + o), make_float4(rn4[0], rn4[1], rn4[2], rn4[3]));
                                        __stcs(reinterpret_cast<float4*>(out2 + o), make_float4(pn4[0], pn4[1], pn4[2], pn4[3]));
                                        __stcs(reinterpret_cast<float4*>(xvec + o), make_float4(xn4[0], xn4[1], xn4[2], xn4[3]));
                                    } else {
#pragma unroll
                                        for (int e = 0; e < 4; e += 2) {
                                            if (gx + e < nx) {   // FP64 rows are only 2-element aligned
                                                if constexpr (!RFOLD)
                                                    *reinterpret_cast<T2*>(out1 + o + e) = T2{rn4[e], rn4[e + 1]};
                                                *reinterpret_cast<T2*>(out2 + o + e) = T2{pn4[e], pn4[e + 1]};
                                                *reinterpret_cast<T2*>(xvec + o + e) = T2{xn4[e], xn4[e + 1]};
                                            }
                                        }
                                    }
                                }
                            }
                        }
                    } else if (MODE == TMODE_RES && interior) {
                        // keep b of this plane for the residual of output plane z
                        T b8[8];
                        load_window<T, 8>(b8, inint + (row - N) * IP + 8 * g);
                        T* rg = ring + rslot * (TY * IP) + (row - N) * IP + 8 * g;
                        if constexpr (sizeof(T) == 4) {
                            reinterpret_cast<float4*>(rg)[0] = make_float4(b8[0], b8[1], b8[2], b8[3]);
                            reinterpret_cast<float4*>(rg)[1] = make_float4(b8[4], b8[5], b8[6], b8[7]);
                        } else {
#pragma unroll
                            for (int e = 0; e < 8; e += 2) *reinterpret_cast<T2*>(rg + e) = T2{b8[e], b8[e + 1]};
                        }
                    }
                    // x-sweep of the 8 outputs as 4 packed pairs (i, i+1); symmetric taps paired.
                    // wp holds v shifted by one so that every operand pair is register-aligned.
                    T2 vp[WIN / 2], wp[WIN / 2 - 1];
#pragma unroll
                    for (int i = 0; i < WIN / 2; i++) vp[i] = T2{v[2 * i], v[2 * i + 1]};
#pragma unroll
                    for (int i = 0; i < WIN / 2 - 1; i++) wp[i] = T2{v[2 * i + 1], v[2 * i + 2]};
                    auto pair_at = [&](int c) -> T2 {   // (v[c], v[c+1])
                        return (c & 1) ? wp[c >> 1] : vp[c >> 1];
                    };
                    T2 mo[4], ko[4];
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        const int cI = HL + i;
                        T2 m = PP::fma(mxp[0], pair_at(cI), PP::zero());
                        T2 k2 = PP::fma(kxp[0], pair_at(cI), PP::zero());
#pragma unroll
                        for (int jj = 1; jj <= N; jj++) {
                            const T2 sp = PP::add(pair_at(cI - jj), pair_at(cI + jj));
                            m = PP::fma(mxp[jj], sp, m);
                            k2 = PP::fma(kxp[jj], sp, k2);
                        }
                        mo[i / 2] = m;
                        ko[i / 2] = k2;
                    }
                    if (zsi != 1) {   // mirrored plane (-1) or a face plane (0)
                        const T2 sg = PP::mk(zsgn);
#pragma unroll
                        for (int i = 0; i < 4; i++) {
                            mo[i] = PP::fma(sg, mo[i], PP::zero());
                            ko[i] = PP::fma(sg, ko[i], PP::zero());
                        }
                    }
                    T* mdst = MXs + row * MXP + 8 * g;
                    T* kdst = KXs + row * MXP + 8 * g;
                    if constexpr (sizeof(T) == 4) {
                        reinterpret_cast<float4*>(mdst)[0] = make_float4(mo[0].x, mo[0].y, mo[1].x, mo[1].y);
                        reinterpret_cast<float4*>(mdst)[1] = make_float4(mo[2].x, mo[2].y, mo[3].x, mo[3].y);
                        reinterpret_cast<float4*>(kdst)[0] = make_float4(ko[0].x, ko[0].y, ko[1].x, ko[1].y);
                        reinterpret_cast<float4*>(kdst)[1] = make_float4(ko[2].x, ko[2].y, ko[3].x, ko[3].y);
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; i++) {
                            *reinterpret_cast<T2*>(mdst + 2 * i) = mo[i];
                            *reinterpret_cast<T2*>(kdst + 2 * i) = ko[i];
                        }
                    }
                }
            }
            __syncthreads();
            if (s_abort) goto abort;
            // the stage is consumed: refill it with plane k + S
            if (tid == 0) {
                if (k + S < np) {
                    fence_proxy_async_smem();
                    issue(k + S);
                }
                if (!BATCH && k == np - 1) fetch();   // next item (a batch fetches after its reduction)
            }
            // ---- y-sweep in registers, then the z push ----
            {
                const int c2 = 2 * lane;
                constexpr int NR = R + 2 * N;
                T2 mv[NR], kv[NR];
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    mv[r] = *reinterpret_cast<const T2*>(mxb + r * MXP);
                    kv[r] = *reinterpret_cast<const T2*>(kxb + r * MXP);
                }
                T2 U[R], V[R], q[R];
#pragma unroll
                for (int t = 0; t < R; t++) {
                    const int cc = t + N;   // centre row in mv/kv
                    T2 u = PP::fma(my[0], mv[cc], PP::zero());
                    T2 w = PP::fma(ky[0], mv[cc], PP::zero());
                    w = PP::fma(my[0], kv[cc], w);
#pragma unroll
                    for (int jj = 1; jj <= N; jj++) {
                        const T2 sm = PP::add(mv[cc - jj], mv[cc + jj]);
                        const T2 sk = PP::add(kv[cc - jj], kv[cc + jj]);
                        u = PP::fma(my[jj], sm, u);
                        w = PP::fma(ky[jj], sm, w);
                        w = PP::fma(my[jj], sk, w);
                    }
                    U[t] = u;
                    V[t] = w;
                }
                push_dispatch<T2, PP, N, R>(jslot, acc, U, V, w1z, mz, q);
                // output plane z - N is complete
                const int zo = z - N;
                if (zo >= z0 && zo < z1) {
                    const int oslot = (zo - z0) % (N + 1);
#pragma unroll
                    for (int t = 0; t < R; t++) {
                        const int gy = y0 + R * warp + t, gx = x0 + c2;
                        if (gy < ny && gx < nx) {
                            const size_t o = ((size_t)zo * ny + gy) * pitch + gx;
                            unsigned mm = 0x0101u;
                            if (!BATCH && a.mbits) {   // gx is even: both bits lie in one word
                                const uint32_t w = a.mbits[((size_t)zo * ny + gy) * a.mwords + (gx >> 5)];
                                const uint32_t pr = (w >> (gx & 31)) & 3u;
                                mm = (pr & 1u) | ((pr & 2u) << 7);   // bytes (x, x + 1) as before
                            }
                            if constexpr (DF && MODE == TMODE_OP) {
                                // y = A x rounded once to FP64
                                const double yx = (mm & 0xffu) ? df_to_double(q[t].x) : 0.0;
                                const double yy = (mm >> 8) ? df_to_double(q[t].y) : 0.0;
                                *reinterpret_cast<double2*>(reinterpret_cast<double*>(out0) + o) = make_double2(yx, yy);
                            } else if constexpr (DF) {
                                // r = b - A x in FP64 from the double-float A x; b is still FP64
                                const double2 bq = *reinterpret_cast<const double2*>(
                                    ring + oslot * (TY * IP) + (R * warp + t) * IP + c2);
                                const double bx = (mm & 0xffu) ? bq.x : 0.0, by = (mm >> 8) ? bq.y : 0.0;
                                const double qx = (mm & 0xffu) ? df_to_double(q[t].x) : 0.0;
                                const double qy = (mm >> 8) ? df_to_double(q[t].y) : 0.0;
                                const double2 r = make_double2(bx - qx, by - qy);
                                *reinterpret_cast<double2*>(reinterpret_cast<double*>(out0) + o) = r;
                                const double wyd = (gx + 1 < nx) ? 1.0 : 0.0;
                                s0 = ::fma(r.x, r.x, ::fma(wyd * r.y, r.y, s0));
                                s1 = ::fma(bx, bx, ::fma(wyd * by, by, s1));
                            } else {
                            const T wy = (gx + 1 < nx) ? T(1) : T(0);   // second of the pair in range?
                            T2 mk2 = PP::mk(T(1));
                            if (mm != 0x0101u) {
                                mk2.x = (mm & 0xffu) ? T(1) : T(0);
                                mk2.y = (mm >> 8) ? T(1) : T(0);
                                q[t].x *= mk2.x;
                                q[t].y *= mk2.y;
                            }
                            if constexpr (MODE == TMODE_OP) {
                                __stcs(reinterpret_cast<T2*>(out0 + o), q[t]);
                            } else {
                                T2 rg = *reinterpret_cast<const T2*>(
                                    ring + oslot * (TY * IP) + (R * warp + t) * IP + c2);
                                if constexpr (MODE == TMODE_RES) {
                                    T2 r;
                                    rg.x *= mk2.x;   // b off the mask is ignored
                                    rg.y *= mk2.y;
                                    r.x = rg.x - q[t].x;
                                    r.y = rg.y - q[t].y;
                                    *reinterpret_cast<T2*>(out0 + o) = r;
                                    d0.add(fma(r.x, r.x, wy * r.y * r.y));
                                    d1.add(fma(rg.x, rg.x, wy * rg.y * rg.y));
                                } else {
                                    __stcs(reinterpret_cast<T2*>(out0 + o), q[t]);
                                    d1.add(fma(rg.x, q[t].x, wy * rg.y * q[t].y));
                                    d2.add(fma(q[t].x, q[t].x, wy * q[t].y * q[t].y));
                                }
                            }
                            }   // not DF
                        }
                    }
                }
            }
            jslot = (jslot + 1 == L) ? 0 : jslot + 1;
            __syncthreads();
        }
        cnt += (uint32_t)np;

        if constexpr (BATCH) {
            // this item's dot products -> its problem's partials; the block finishing the
            // problem's last item adds them in item order and runs the CG finaliser
            double v3[3] = {d0.value(), d1.value(), d2.value()};
            d0 = KSum<T>();
            d1 = KSum<T>();
            d2 = KSum<T>();
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                const double t = warp_sum(v3[kk]);
                if (lane == 0) s_red[kk * (kTNT / 32) + warp] = t;
            }
            __syncthreads();
            const BatchProblem<T>& P = probs[cur_prob];
            if (tid == 0) {
                for (int kk = 0; kk < 3; kk++) {
                    double t = 0.0;
                    for (int w = 0; w < kTNT / 32; w++) t += s_red[kk * (kTNT / 32) + w];
                    P.partials[3 * item + kk] = t;
                }
                __threadfence();
                const unsigned prev = atomicAdd(P.items_done, 1u);
                s_last = (prev + 1 == (unsigned)P.nitems);
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                double acc3[3] = {0.0, 0.0, 0.0};
                for (int i = tid; i < P.nitems; i += kTNT)
#pragma unroll
                    for (int kk = 0; kk < 3; kk++) acc3[kk] += __ldcg(P.partials + 3 * i + kk);
#pragma unroll
                for (int kk = 0; kk < 3; kk++) {
                    const double t = warp_sum(acc3[kk]);
                    if (lane == 0) s_red[kk * (kTNT / 32) + warp] = t;
                }
                __syncthreads();
                if (tid == 0) {
                    double tot[3];
                    for (int kk = 0; kk < 3; kk++) {
                        tot[kk] = 0.0;
                        for (int w = 0; w < kTNT / 32; w++) tot[kk] += s_red[kk * (kTNT / 32) + w];
                    }
                    if (!P.timing) finalize_cg1(P.sc, tot[0], tot[1], tot[2]);
                    *P.items_done = 0;
                    __threadfence();
                }
            }
            if (tid == 0) fetch();
            __syncthreads();
        }
    }

    // every block: count itself out; the last one resets the work counters for the next launch
    if (tid == 0) {
        __threadfence();
        const unsigned done_blocks = atomicAdd(&a.work[1], 1u) + 1;
        if (done_blocks == gridDim.x) {
            a.work[0] = 0;
            a.work[1] = 0;
            __threadfence();
        }
    }
    if (!BATCH && a.fin != FIN_NONE) {
        if constexpr (MODE == TMODE_CG) {
            double v3[3] = {d0.value(), d1.value(), d2.value()};
            grid_reduce_k<kTNT, 3>(v3, a.partials, a.sc, a.fin);
        } else if constexpr (DF) {
            double v2[2] = {s0, s1};
            grid_reduce_k<kTNT, 2>(v2, a.partials, a.sc, a.fin);
        } else {
            double v2[2] = {d0.value(), d1.value()};
            grid_reduce_k<kTNT, 2>(v2, a.partials, a.sc, a.fin);
        }
    }
    return;

abort:
    // A TMA load did not complete within the time limit: report it, give the loads still in
    // flight a bounded time to land (they target this block's shared memory), and stop. The
    // work counters are left as they are; the host resets them before the next solve.
    if (tid == 0) {
        atomicExch(&a.sc->status, -4);
        atomicExch(&a.sc->done, 1);
        __threadfence();
        for (uint32_t i = s_wait_from; i < s_issued; i++)
            mbar_wait_bounded(&bars[i % S], (i / S) & 1u, 100000000ull);
    }
}

}  // namespace bsk

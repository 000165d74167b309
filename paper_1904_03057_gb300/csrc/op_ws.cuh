// op_ws.cuh -- warp-specialised FP32 passes for unmasked box problems whose rows are 16-byte
// multiples (TMA-addressable), degrees 1..4: the operator y = A x (WS_OP) and one whole CG
// iteration in a single pass (WS_CG).
//
// The operator (arXiv:1904.03057 section 2.4, Eq. tensForm with constant coefficients; the
// separable chains of Fig. FiltAlg) is applied as
//     A x = (Mz + dt Kz) U + Mz V,    U = My MX,    V = dt Ky MX + My KX,
//     MX = Mx x,    KX = dt Kx x,
// seven band convolutions of 2n+1 taps per unknown, with odd reflection of the coefficients at
// the box faces (c_{-i} = -c_i, c_0 = 0 in 1-based numbering, the same at N+1). On an isotropic
// grid (hx = hy = hz) My = Mz and dt Ky = dt Kz, and the z step is taken as
// Mz (U + V) + dt Kz U, so that the y/z threads hold two tap sets instead of four.
//
// A block owns a 64 x 32 (x, y) output tile and marches along z; 16 warps, four per SM
// sub-partition, in three roles:
//   x warps (0-3)  -- one tile row per lane, 16 columns per warp: wait for the plane's TMA box
//                     (tile plus n rows and 4 columns of halo), complete the face ghosts by odd
//                     reflection in registers (a ghost row reads its mirror row, ghost columns
//                     are rebuilt in the loaded window) and run the x-sweep, writing MX and KX
//                     into one of two shared-memory buffers. In CG mode the boxes hold p_{m-1},
//                     q_{m-1} and p_{m-2}; the window first becomes r_{m-1} = p_{m-1} -
//                     beta_{m-2} p_{m-2} (no r is stored), then r_m = r_{m-1} - alpha q_{m-1}
//                     and the new search direction p_m = r_m + beta p_{m-1}, and the lane writes
//                     p and x = x + alpha p_{m-1} of its interior row to HBM and reduces r.r.
//   halo warps (4-7) -- the same x-sweep for the 2n halo rows of the box, 8 columns per lane;
//                     lane 0 of warp 4 also issues the TMA loads into a stage ring, refilling a
//                     stage once every x thread has released it.
//   y/z warps (8-15) -- each lane owns two columns and four rows: it reads its 2n+4 rows of MX
//                     and KX, forms U and V for its four rows (y-sweep) and pushes them, with the
//                     2n+1 z taps, into a register ring of accumulators for output planes
//                     z-n .. z+n; output plane z-n is then complete and leaves to HBM (CG: as
//                     q = A p, with p.q and q.q reduced).
// The roles hand the stages and the x-sweep buffers over through mbarriers only; no block-wide
// barrier separates the phases of a plane. Every wait is bounded in time; a wait that gives up
// raises a block flag that makes every other wait give up too, and the block reports status -4.
// Blocks are persistent (one per SM) and take (tile, z-chunk) items round-robin; the TMA issuer
// runs ahead across item boundaries.
#pragma once

#include <type_traits>

#include "bsk_device.cuh"
#include "tma_util.cuh"

namespace bsk {

constexpr int kWsTX = 64;     // output columns per tile (32 lanes x 2)
constexpr int kWsTY = 32;     // output rows per tile (one per x-warp lane)
constexpr int kWsR = 4;       // output rows per y/z thread
constexpr int kWsWX = 4;      // x warps
constexpr int kWsWH = 4;      // halo warps
constexpr int kWsWY = 8;      // y/z warps
constexpr int kWsNT = 32 * (kWsWX + kWsWH + kWsWY);

enum WsMode : int { WS_OP = 0, WS_CG = 1 };

template <int N, int MODE>
struct WsGeo {
    static_assert(N >= 1 && N <= 4, "the x window carries four halo columns");
    static constexpr int L = 2 * N + 1;
    static constexpr int HL = 4;                    // halo columns staged on each side
    static constexpr int BX = kWsTX + 2 * HL + 4;   // box width; rows 76 floats apart put the 16-byte
                                                    // loads of consecutive rows in distinct banks
    static constexpr int HY = kWsTY + 2 * N;        // box height
    static constexpr int MXP = kWsTX + 4;           // row pitch of MX, KX
    static constexpr int NXT = 32 * (kWsWX + kWsWH);   // x and halo threads
    static constexpr int NYZ = 32 * kWsWY;
    static constexpr int NIN = MODE == WS_CG ? 3 : 1;   // halo boxes per stage: x, or r, q, p
    // TMA stages: as many as shared memory allows the CG pass; 8 (a power of two, so the stage
    // index and parity are a mask and a shift) for the operator, which measured 2 % faster than 6
    static constexpr int S = MODE == WS_CG ? (N >= 4 ? 3 : 4) : 8;
    static constexpr int D = 2;                         // MX / KX buffers
    static constexpr size_t rnd(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t box_bytes = rnd(sizeof(float) * HY * BX);
    // CG: interior box of x with rows of IP = 68 floats (64 used), so that the x lanes (one row
    // each) hit distinct shared-memory banks with their 16-byte loads
    static constexpr int IP = kWsTX + 4;
    static constexpr size_t int_bytes = sizeof(float) * IP * kWsTY;
    static constexpr size_t stage_bytes = NIN * box_bytes + (MODE == WS_CG ? int_bytes : 0);
    static constexpr size_t mx_bytes = rnd(sizeof(float) * HY * MXP);
    static constexpr size_t off_mx = S * stage_bytes;
    static constexpr size_t off_bar = off_mx + 2 * D * mx_bytes;
    static constexpr size_t total = off_bar + 8 * (2 * S + 2 * D);
    // bytes the TMA loads of one stage deliver (the boxes themselves, not their rounded slots)
    static constexpr uint32_t tx_bytes =
        (uint32_t)(NIN * sizeof(float) * HY * BX + (MODE == WS_CG ? int_bytes : 0));
    static_assert(total <= 220 * 1024, "shared memory budget");
};

struct WsArgs {
    CUtensorMap tin[3];   // halo boxes (BX, HY, 1): OP {x}; CG {p_{m-1}, q_{m-1}, p_{m-2}}
    CUtensorMap tint;     // CG: interior box (68, 32, 1) of x (64 columns used)
    float* out0;          // OP y; CG q = A p
    float* out1;          // unused (CG keeps no r)
    float* out2;          // CG p
    float* xvec;          // CG x, updated in place
    Scalars* sc;          // CG scalars; OP: receives status -4 on a wait time-out (may be null)
    double* partials;     // CG: 3 doubles per block
    int fin;              // CG: FIN_CG1 or FIN_NORM; OP: FIN_NONE
    int nx, ny, nz;       // rows are nx floats (a multiple of 4)
    int tiles_x, tiles_y, tz, nitems;
    float M[3][kMaxTaps];   // per-axis mass kernels, index j + n
    float K[3][kMaxTaps];   // per-axis stiffness kernels times dt
};

// Bounded wait on an mbarrier phase that also gives up once another thread has raised the
// block's abort flag. On a time-out it raises the flag itself.
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        for (int i = 0; i < 32; i++)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (global_timer_ns() - t0 > 2000000000ull) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void ws_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Ghost columns of a window v[0..W) whose element i is grid column x0 - 4 + col0 + i.
// Low face (x0 = 0, col0 = 0): column -1 is the face (zero), column -1-j mirrors j-1 with a sign.
template <int W>
__device__ __forceinline__ void ws_fix_lo(float (&v)[W])
{
    v[3] = 0.f;
    v[2] = -v[4];
    v[1] = -v[5];
    v[0] = -v[6];
}
// High face at window position P (grid column nx): zero there, nx+j mirrors nx-j with a sign.
template <int W, int P, int N>
__device__ __forceinline__ void ws_fix_hi_p(float (&v)[W])
{
    v[P] = 0.f;
#pragma unroll
    for (int j = 1; j <= N; j++)
        if (P + j < W) v[P + j] = -v[P - j];
}
// The window positions a face can take where it matters: stored outputs sit at 4..W-5, and with
// nx, x0 and col0 multiples of 4 the face lies at a multiple of 4 (0 = no face in reach).
template <int W, int N>
__device__ __forceinline__ void ws_fix_hi(float (&v)[W], int p)
{
    switch (p) {
    case 8: ws_fix_hi_p<W, 8, N>(v); break;
    case 12: if constexpr (W > 12) ws_fix_hi_p<W, 12, N>(v); break;
    case 16: if constexpr (W > 16) ws_fix_hi_p<W, 16, N>(v); break;
    case 20: if constexpr (W > 20) ws_fix_hi_p<W, 20, N>(v); break;
    default: break;
    }
}

// Interior bookkeeping of one x task in CG mode (z inside the item, row and columns inside the
// grid): write p and x of the 16 outputs and add r.r. p is stored with the default cache
// policy: the y/z threads of the block read it back from L2 n planes later for p.q. On the
// large grids measured this beat keeping a ring of p planes in shared memory, whose space now
// holds one more TMA stage.
struct WsCgOut {
    float* p;
    float* x;
    const float4* xin;      // x of the 16 outputs (interior box in shared memory)
    int ncols;              // columns of the 16 inside the grid (multiple of 4 at most 16)
};

// x-sweep of G outputs of one box row from a 16-byte aligned window of G + 8 floats of each input
// box. OP: the window is x. CG: the window is p_new = (r - alpha q) + beta p_old with
// r = p_old - beta_prev p_older rebuilt from the boxes (p_old, q, p_older), and (G = 16 with `co`
// set) the lane also stores p, x of its interior outputs. MX, KX of the G outputs are scaled by sgn (row sign x plane sign) when it is not 1.
template <int N, int G, int MODE>
__device__ __forceinline__ void ws_x(const float* src0, const float* src1, const float* src2, float* mdst,
                                     float* kdst, const float2 (&mxp)[N + 1], const float2 (&kxp)[N + 1],
                                     float sgn, bool lo, int hip, float alpha, float beta, float beta_prev,
                                     const WsCgOut* co,
                                     float& rr_part, uint64_t* release)
{
    constexpr int W = G + 8;
    float v[W];
#pragma unroll
    for (int qd = 0; qd < W / 4; qd++) {
        const float4 f = reinterpret_cast<const float4*>(src0)[qd];
        if constexpr (MODE == WS_CG) {
            const float4 fq = reinterpret_cast<const float4*>(src1)[qd];
            const float4 fp = reinterpret_cast<const float4*>(src2)[qd];
            const float po[4] = {f.x, f.y, f.z, f.w};   // p_{m-1}
            const float rn[4] = {fmaf(-alpha, fq.x, fmaf(-beta_prev, fp.x, f.x)),
                                 fmaf(-alpha, fq.y, fmaf(-beta_prev, fp.y, f.y)),
                                 fmaf(-alpha, fq.z, fmaf(-beta_prev, fp.z, f.z)),
                                 fmaf(-alpha, fq.w, fmaf(-beta_prev, fp.w, f.w))};
#pragma unroll
            for (int e = 0; e < 4; e++) v[4 * qd + e] = fmaf(beta, po[e], rn[e]);
            // interior outputs occupy window positions 4 .. 4 + G - 1 (chunks 1 .. G/4)
            if (co && qd >= 1 && qd <= G / 4 && 4 * (qd - 1) < co->ncols) {
                const int o = 4 * (qd - 1);
                const float4 xi = co->xin[qd - 1];
                const float4 pn = make_float4(v[4 * qd], v[4 * qd + 1], v[4 * qd + 2], v[4 * qd + 3]);
                *reinterpret_cast<float4*>(co->p + o) = pn;
                __stcs(reinterpret_cast<float4*>(co->x + o),
                       make_float4(fmaf(alpha, po[0], xi.x), fmaf(alpha, po[1], xi.y), fmaf(alpha, po[2], xi.z),
                                   fmaf(alpha, po[3], xi.w)));

                rr_part = fmaf(rn[0], rn[0], rr_part);
                rr_part = fmaf(rn[1], rn[1], rr_part);
                rr_part = fmaf(rn[2], rn[2], rr_part);
                rr_part = fmaf(rn[3], rn[3], rr_part);
            }
        } else {
            v[4 * qd] = f.x; v[4 * qd + 1] = f.y; v[4 * qd + 2] = f.z; v[4 * qd + 3] = f.w;
        }
    }
    // the stage is no longer read by this thread: release it now, ahead of the arithmetic, so the
    // issuer can refill it as early as possible
    ws_arrive(release);
    if (lo) ws_fix_lo<W>(v);
    if (hip) ws_fix_hi<W, N>(v, hip);
    auto P = [&](int s) { return make_float2(v[s], v[s + 1]); };
    const bool flip = sgn != 1.f;   // a mirrored row or plane (-1), or a face (0)
    const float2 sg = make_float2(sgn, sgn);
#pragma unroll
    for (int i = 0; i < G / 2; i += 2) {
        float2 m2[2], k2[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int w = 4 + 2 * (i + h);
            float2 m = __fmul2_rn(mxp[0], P(w));
            float2 k = __fmul2_rn(kxp[0], P(w));
#pragma unroll
            for (int j = 1; j <= N; j++) {
                const float2 sp = __fadd2_rn(P(w - j), P(w + j));
                m = __ffma2_rn(mxp[j], sp, m);
                k = __ffma2_rn(kxp[j], sp, k);
            }
            if (flip) {
                m = __fmul2_rn(sg, m);
                k = __fmul2_rn(sg, k);
            }
            m2[h] = m;
            k2[h] = k;
        }
        reinterpret_cast<float4*>(mdst)[i / 2] = make_float4(m2[0].x, m2[0].y, m2[1].x, m2[1].y);
        reinterpret_cast<float4*>(kdst)[i / 2] = make_float4(k2[0].x, k2[0].y, k2[1].x, k2[1].y);
    }
}

// z push of the four rows into the accumulator ring (slot of output plane z + d is (J + d) mod L),
// handing back the completed output plane z - n and clearing its slot. The ring receives
// c1[|d|] A + c2[|d|] B: (W1z, Mz) on (U, V), or on an isotropic grid (Mz, dt Kz) on (U + V, U).
template <int N, int J>
__device__ __forceinline__ void ws_push(float2 (&acc)[kWsR][2 * N + 1], const float2 (&A)[kWsR],
                                        const float2 (&B)[kWsR], const float2 (&c1)[N + 1],
                                        const float2 (&c2)[N + 1], float2 (&q)[kWsR])
{
    constexpr int L = 2 * N + 1;
#pragma unroll
    for (int t = 0; t < kWsR; t++) {
#pragma unroll
        for (int dd = -N; dd <= N; dd++) {
            const int sl = ((J + dd) % L + L) % L;
            const int ad = dd < 0 ? -dd : dd;
            acc[t][sl] = __ffma2_rn(c1[ad], A[t], acc[t][sl]);
            acc[t][sl] = __ffma2_rn(c2[ad], B[t], acc[t][sl]);
        }
        constexpr int fs = ((J - N) % L + L) % L;
        q[t] = acc[t][fs];
        acc[t][fs] = make_float2(0.f, 0.f);
    }
}

template <int N>
__device__ __forceinline__ void ws_push_dispatch(int j, float2 (&acc)[kWsR][2 * N + 1], const float2 (&A)[kWsR],
                                                 const float2 (&B)[kWsR], const float2 (&c1)[N + 1],
                                                 const float2 (&c2)[N + 1], float2 (&q)[kWsR])
{
    switch (j) {
    case 0: ws_push<N, 0>(acc, A, B, c1, c2, q); break;
    case 1: ws_push<N, 1>(acc, A, B, c1, c2, q); break;
    case 2: ws_push<N, 2>(acc, A, B, c1, c2, q); break;
    default:
        if constexpr (N >= 2) {
            switch (j) {
            case 3: ws_push<N, 3>(acc, A, B, c1, c2, q); break;
            case 4: ws_push<N, 4>(acc, A, B, c1, c2, q); break;
            default:
                if constexpr (N >= 3) {
                    switch (j) {
                    case 5: ws_push<N, 5>(acc, A, B, c1, c2, q); break;
                    case 6: ws_push<N, 6>(acc, A, B, c1, c2, q); break;
                    default:
                        if constexpr (N >= 4) {
                            if (j == 7) ws_push<N, 7>(acc, A, B, c1, c2, q);
                            else ws_push<N, 8>(acc, A, B, c1, c2, q);
                        }
                    }
                }
            }
        }
    }
}

// Planes k + J, J = 0 .. L - 1 (those below np) of a y/z thread's march, each with its
// compile-time accumulator slot J; false as soon as one step reports a wait that gave up.
template <int J, int L, typename F>
__device__ __forceinline__ bool ws_unroll_planes(F& step, int k, int np)
{
    if constexpr (J < L) {
        if (k + J >= np) return true;
        if (!step(k + J, std::integral_constant<int, J>{})) return false;
        return ws_unroll_planes<J + 1, L>(step, k, np);
    } else {
        return true;
    }
}

// Compensated (Kahan) FP32 running sum, converted to FP64 once per thread.
struct WsKSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <int N, int MODE, bool ISO>
__global__ void __launch_bounds__(kWsNT, 1) k_ws(const __grid_constant__ WsArgs a)
{
    using G = WsGeo<N, MODE>;
    constexpr int L = G::L, S = G::S, D = G::D, HY = G::HY, BX = G::BX, MXP = G::MXP, HL = G::HL;
    constexpr bool CG = MODE == WS_CG;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + G::off_bar);
    uint64_t* empty = full + S;
    uint64_t* mxfull = empty + S;
    uint64_t* mxempty = mxfull + D;
    __shared__ int s_abort;
    __shared__ uint32_t s_issued;   // planes whose loads the issuer has started
    volatile int* abort_flag = &s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (CG) {
        if (*(volatile int*)&a.sc->done) return;   // uniform over the grid
    }
    const int ntiles = a.tiles_x * a.tiles_y;
    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], G::NXT);
        }
        for (int d = 0; d < D; d++) {
            mbar_init(&mxfull[d], G::NXT);
            mbar_init(&mxempty[d], G::NYZ);
        }
        fence_mbar_init();
        s_abort = 0;
        s_issued = 0;
    }
    __syncthreads();

    auto item_geo = [&](int item, int& x0, int& y0, int& z0, int& z1) {
        const int tile = item % ntiles, zc = item / ntiles;
        x0 = (tile % a.tiles_x) * kWsTX;
        y0 = (tile / a.tiles_x) * kWsTY;
        z0 = zc * a.tz;
        z1 = min(z0 + a.tz, a.nz);
    };
    auto mx_buf = [&](int d) { return reinterpret_cast<float*>(smem + G::off_mx + 2 * d * G::mx_bytes); };
    auto kx_buf = [&](int d) { return reinterpret_cast<float*>(smem + G::off_mx + (2 * d + 1) * G::mx_bytes); };
    float alpha = 0.f, beta = 0.f, beta_prev = 0.f;
    if (CG) {
        alpha = (float)a.sc->alpha;
        beta = (float)a.sc->beta;
        beta_prev = (float)a.sc->beta_prev;
    }
    WsKSum d0, d1, d2;   // CG: r.r (x warps), p.q and q.q (y/z warps)
    uint32_t c = 0;      // planes consumed by this thread's role

    if (warp < kWsWX + kWsWH) {
        // ------------------------------------------------------------ x and halo warps
        const bool is_x = warp < kWsWX;
        const int wq = warp & 3;
        float2 mxp[N + 1], kxp[N + 1];
#pragma unroll
        for (int j = 0; j <= N; j++) {
            mxp[j] = make_float2(a.M[0][N + j], a.M[0][N + j]);
            kxp[j] = make_float2(a.K[0][N + j], a.K[0][N + j]);
        }
        // x warps: box row N + lane, columns 16 wq ..; halo warps: one of 16 N tasks of 8 columns
        // of the 2N halo rows (rows 0..N-1 and N+32..2N+31), lanes < 4N, consecutive lanes on
        // consecutive rows (distinct banks)
        const int hb = wq * 4 * N + lane;
        const bool task = is_x || lane < 4 * N;
        const int hrow = hb % (2 * N);
        const int br = is_x ? N + lane : (hrow < N ? hrow : hrow + kWsTY);
        const int col = is_x ? 16 * wq : 8 * (hb / (2 * N));

        // TMA issuer (lane 0 of the first halo warp): the next plane to load, across items
        const bool issuer = warp == kWsWX && lane == 0;
        int p_item = blockIdx.x, p_k = 0, p_np = 0, p_x0 = 0, p_y0 = 0, p_z0 = 0;
        uint32_t p_c = 0;
        auto p_setup = [&]() {
            if (p_item < a.nitems) {
                int z1;
                item_geo(p_item, p_x0, p_y0, p_z0, z1);
                p_np = z1 - p_z0 + 2 * N;
            }
        };
        auto issue_next = [&]() {
            if (p_item >= a.nitems) return;
            const int zz = p_z0 - N + p_k;
            int zsrc = 0;
            if (!reflect_index(zz, a.nz, zsrc)) zsrc = 0;   // a face plane: any plane, scaled by 0
            const int st = (int)(p_c % S);
            unsigned char* base = smem + st * G::stage_bytes;
            mbar_arrive_expect_tx(&full[st], G::tx_bytes);
#pragma unroll
            for (int i = 0; i < G::NIN; i++)
                tma_load_3d(base + i * G::box_bytes, &a.tin[i], &full[st], p_x0 - HL, p_y0 - N, zsrc);
            if (CG)   // the interior x of the plane (halo planes: any plane, unused)
                tma_load_3d(base + G::NIN * G::box_bytes, &a.tint, &full[st], p_x0, p_y0,
                            min(max(zz, 0), a.nz - 1));
            p_c++;
            s_issued = p_c;
            if (++p_k == p_np) {
                p_item += gridDim.x;
                p_k = 0;
                p_setup();
            }
        };
        if (issuer) {
            for (int i = 0; i < G::NIN; i++) prefetch_tensormap(&a.tin[i]);
            if (CG) prefetch_tensormap(&a.tint);
            p_setup();
            for (int k = 0; k < S; k++) issue_next();
        }

        float rr_part = 0.f;
        bool stop = false;
        for (int item = blockIdx.x; item < a.nitems && !stop; item += gridDim.x) {
            int x0, y0, z0, z1;
            item_geo(item, x0, y0, z0, z1);
            const int np = z1 - z0 + 2 * N;
            // this lane's box row: its source (the mirror row for a ghost) and sign
            int sy = 0;
            const int gy = y0 - N + br;
            const int rs = reflect_index(gy, a.ny, sy);
            int src = sy - (y0 - N);
            float rsg = (float)rs;
            if (rs == 0 || src < 0 || src >= HY) {
                src = br;
                rsg = 0.f;
            }
            const bool lo = x0 == 0 && col == 0;
            constexpr int WIN = 16 + 8;
            int hip = a.nx - (x0 - HL + col);
            hip = (hip >= 5 && hip < (is_x ? WIN : 16)) ? hip : 0;
            // CG interior: a real row of the grid, columns inside it
            const bool interior_row = CG && is_x && rs == 1;
            const int ncols = min(16, a.nx - (x0 + col));
            const size_t rowoff = (size_t)(y0 + lane) * a.nx + x0 + col;
            const size_t planesz = (size_t)a.nx * a.ny;
            for (int k = 0; k < np; k++, c++) {
                const int st = (int)(c % S), d = (int)(c % D);
                if (!ws_wait(&full[st], (c / S) & 1u, abort_flag)) { stop = true; break; }
                if (c >= (uint32_t)D && !ws_wait(&mxempty[d], ((c / D) - 1) & 1u, abort_flag)) {
                    stop = true;
                    break;
                }
                const int z = z0 - N + k;
                int zsrc = 0;
                const float zsg = (float)reflect_index(z, a.nz, zsrc);
                const unsigned char* base = smem + st * G::stage_bytes;
                const float* b0 = reinterpret_cast<const float*>(base) + src * BX + col;
                const float* b1 = reinterpret_cast<const float*>(base + G::box_bytes) + src * BX + col;
                const float* b2 = reinterpret_cast<const float*>(base + 2 * G::box_bytes) + src * BX + col;
                float* md = mx_buf(d) + br * MXP + col;
                float* kd = kx_buf(d) + br * MXP + col;
                if (task) {
                    if (is_x) {
                        WsCgOut co;
                        const bool inz = z >= z0 && z < z1;

                        if (CG && interior_row && inz && ncols > 0) {
                            const size_t o = (size_t)z * planesz + rowoff;
                            co.p = a.out2 + o;
                            co.x = a.xvec + o;
                            co.xin = reinterpret_cast<const float4*>(
                                reinterpret_cast<const float*>(base + G::NIN * G::box_bytes) + lane * G::IP + col);
                            co.ncols = ncols;
                        }
                        ws_x<N, 16, MODE>(b0, b1, b2, md, kd, mxp, kxp, zsg * rsg, lo, hip, alpha, beta,
                                          beta_prev, (CG && interior_row && inz && ncols > 0) ? &co : nullptr, rr_part,
                                          &empty[st]);
                    } else {
                        ws_x<N, 8, MODE>(b0, b1, b2, md, kd, mxp, kxp, zsg * rsg, lo, hip, alpha, beta, beta_prev, nullptr,
                                         rr_part, &empty[st]);
                    }
                } else {
                    ws_arrive(&empty[st]);
                }
                ws_arrive(&mxfull[d]);
                if (issuer) {
                    // every x thread has released this plane's stage: refill it with plane c + S
                    if (!ws_wait(&empty[st], (c / S) & 1u, abort_flag)) { stop = true; break; }
                    issue_next();
                }
            }
        }
        if (CG) d0.add(rr_part);
    } else {
        // ------------------------------------------------------------ y/z warps
        const int r0 = (warp - kWsWX - kWsWH) * kWsR;   // first tile row of this lane
        const int c2 = 2 * lane;
        float2 my[N + 1], ky[N + 1];
        float2 c1[N + 1], c2t[N + 1];   // z taps applied to (A, B) in the push
#pragma unroll
        for (int j = 0; j <= N; j++) {
            my[j] = make_float2(a.M[1][N + j], a.M[1][N + j]);
            ky[j] = make_float2(a.K[1][N + j], a.K[1][N + j]);
            if constexpr (!ISO) {
                const float w = a.M[2][N + j] + a.K[2][N + j];
                c1[j] = make_float2(w, w);
                c2t[j] = make_float2(a.M[2][N + j], a.M[2][N + j]);
            }
        }
        const size_t plane = (size_t)a.nx * a.ny;
        bool stop = false;
        for (int item = blockIdx.x; item < a.nitems && !stop; item += gridDim.x) {
            int x0, y0, z0, z1;
            item_geo(item, x0, y0, z0, z1);
            const int np = z1 - z0 + 2 * N;
            const int gy0 = y0 + r0, gx = x0 + c2;
            const int nrows = min(kWsR, a.ny - gy0);   // rows of this lane inside the grid
            const bool colok = gx < a.nx;
            float* obase = a.out0 + (size_t)gy0 * a.nx + gx;
            float2 acc[kWsR][L];
#pragma unroll
            for (int t = 0; t < kWsR; t++)
#pragma unroll
                for (int s = 0; s < L; s++) acc[t][s] = make_float2(0.f, 0.f);
            // one input plane; its accumulator slot (k mod L, as every item starts at slot 0) is
            // either a compile-time constant (the operator's plane loop is unrolled by L) or a
            // runtime index (the CG pass and degree 4, whose unrolled forms spilled); false: a
            // wait gave up
            auto plane_step = [&](int k, auto jc) -> bool {
                const int d = (int)(c % D);
                if (!ws_wait(&mxfull[d], (c / D) & 1u, abort_flag)) return false;
                const float* mxb = mx_buf(d) + r0 * MXP + c2;
                const float* kxb = kx_buf(d) + r0 * MXP + c2;
                const int zo = z0 - 2 * N + k;   // output plane completed by this input plane
                float2 pv[kWsR];
                if (CG && zo >= z0 && colok) {
                    // p of the output plane: written by this block's x threads n planes ago (before
                    // their mxfull arrivals, which this thread has acquired) and still in L2
                    const float* pg = a.out2 + (size_t)zo * plane + (size_t)gy0 * a.nx + gx;
#pragma unroll
                    for (int t = 0; t < kWsR; t++)
                        pv[t] = t < nrows ? *reinterpret_cast<const float2*>(pg + (size_t)t * a.nx) : make_float2(0.f, 0.f);
                }
                float2 A[kWsR], B[kWsR];
                {
                    constexpr int NR = kWsR + 2 * N;
                    float2 mv[NR], kv[NR];
#pragma unroll
                    for (int r = 0; r < NR; r++) {
                        mv[r] = *reinterpret_cast<const float2*>(mxb + r * MXP);
                        kv[r] = *reinterpret_cast<const float2*>(kxb + r * MXP);
                    }
#pragma unroll
                    for (int t = 0; t < kWsR; t++) {
                        const int cc = t + N;
                        float2 u = __fmul2_rn(my[0], mv[cc]);
                        float2 w = __fmul2_rn(ky[0], mv[cc]);
                        w = __ffma2_rn(my[0], kv[cc], w);
#pragma unroll
                        for (int jj = 1; jj <= N; jj++) {
                            const float2 sm = __fadd2_rn(mv[cc - jj], mv[cc + jj]);
                            const float2 sk = __fadd2_rn(kv[cc - jj], kv[cc + jj]);
                            u = __ffma2_rn(my[jj], sm, u);
                            w = __ffma2_rn(ky[jj], sm, w);
                            w = __ffma2_rn(my[jj], sk, w);
                        }
                        if constexpr (ISO) {   // (Mz, dt Kz) = (My, dt Ky) on (U + V, U)
                            A[t] = __fadd2_rn(u, w);
                            B[t] = u;
                        } else {               // (W1z, Mz) on (U, V)
                            A[t] = u;
                            B[t] = w;
                        }
                    }
                }
                ws_arrive(&mxempty[d]);
                float2 q[kWsR];
                if constexpr (std::is_integral<decltype(jc)>::value) {
                    if constexpr (ISO) ws_push_dispatch<N>(jc, acc, A, B, my, ky, q);
                    else ws_push_dispatch<N>(jc, acc, A, B, c1, c2t, q);
                } else {
                    constexpr int J = decltype(jc)::value;
                    if constexpr (ISO) ws_push<N, J>(acc, A, B, my, ky, q);
                    else ws_push<N, J>(acc, A, B, c1, c2t, q);
                }
                if (zo >= z0 && colok) {
                    float* o = obase + (size_t)zo * plane;
#pragma unroll
                    for (int t = 0; t < kWsR; t++)
                        if (t < nrows) {
                            __stcs(reinterpret_cast<float2*>(o + (size_t)t * a.nx), q[t]);
                            if (CG) {
                                d1.add(fmaf(pv[t].x, q[t].x, pv[t].y * q[t].y));
                                d2.add(fmaf(q[t].x, q[t].x, q[t].y * q[t].y));
                            }
                        }
                }
                c++;
                return true;
            };
            if constexpr (MODE == WS_OP && N <= 3) {   // degree 4 spilled when unrolled
                for (int k = 0; k < np; k += L)
                    if (!ws_unroll_planes<0, L>(plane_step, k, np)) {
                        stop = true;
                        break;
                    }
            } else {
                int jslot = 0;
                for (int k = 0; k < np; k++) {
                    if (!plane_step(k, jslot)) {
                        stop = true;
                        break;
                    }
                    jslot = (jslot + 1 == L) ? 0 : jslot + 1;
                }
            }
        }
    }

    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            // a wait gave up: report it and give the loads still in flight (they target this
            // block's shared memory) a bounded time to land
            if (a.sc) {
                atomicExch(&a.sc->status, -4);
                atomicExch(&a.sc->done, 1);
                __threadfence();
            }
            const uint32_t issued = s_issued;
            for (uint32_t i = (issued > (uint32_t)S ? issued - S : 0); i < issued; i++)
                mbar_wait_bounded(&full[i % S], (i / S) & 1u, 100000000ull);
        }
        return;   // uniform: s_abort is read after the barrier
    }
    if (CG && a.fin != FIN_NONE) {
        double v3[3] = {d0.value(), d1.value(), d2.value()};
        grid_reduce_k<kWsNT, 3>(v3, a.partials, a.sc, a.fin);
    }
}

}  // namespace bsk

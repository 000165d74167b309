// FP32 instantiation of the TMA operator / single-pass CG kernels (degrees 1..5).
#include <cstring>
#define BSK_T float
#define BSK_TMA_HIGH_DEGREE 1
#include "tma_impl.cuh"

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

// One thread per 32-bit word of the bit-packed mask: bit i of word w of row (z, y) is node
// x = 32 w + i of that row (rows padded to whole words with zero bits).
__global__ void k_pack_mask(const uint8_t* __restrict__ mask, int nx, long long rows, int words,
                            uint32_t* __restrict__ bits)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * words) return;
    const long long row = t / words;
    const int w = (int)(t - row * words);
    const uint8_t* src = mask + row * nx + 32 * w;
    const int n = min(32, nx - 32 * w);
    uint32_t v = 0u;
    for (int i = 0; i < n; i++) v |= (src[i] != 0 ? 1u : 0u) << i;
    bits[t] = v;
}

}  // namespace

int mask_words(int nx) { return (nx + 31) / 32; }

cudaError_t launch_pack_mask(const uint8_t* mask, int nx, int ny, int nz, uint32_t* bits, cudaStream_t s)
{
    const long long rows = (long long)ny * nz;
    const int words = mask_words(nx);
    const long long n = rows * words;
    k_pack_mask<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mask, nx, rows, words, bits);
    return cudaGetLastError();
}

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

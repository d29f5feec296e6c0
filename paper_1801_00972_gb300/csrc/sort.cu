// Periodic counting sort of one species (histogram, exclusive scan, scatter),
// dropping dead slots.  The FP64 path sorts by linear cell index; the mixed
// path by tile (blocks of tile[0] x tile[1] x tile[2] cells, tile-major, the
// cells of a tile row-major inside it), so that each tile's particles occupy
// one contiguous slot range, which the push hands to one thread block.  The
// order of particles inside a cell is not fixed (atomic scatter); nothing in a
// step depends on it: the deposit is an exact integer sum and the random
// numbers are keyed on particle ids.
#include <algorithm>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;
constexpr int kScanBlock = kScanThreads * kScanPer;

// sort key geometry: tiles of tx x ty x tz cells, ntx x nty tiles per plane;
// order: 0 one key per cell, 1 one key per tile (no order inside it), 2 one key
// per block of 2 x 2 x 2 cells inside the tile
struct KeyGeo {
    int tx, ty, tz, ntx, nty, order;
};

// mixed: tile index * (cells per tile) + the cell's row-major index inside its
// tile (or of its block of 2 x 2 x 2 cells, or only the tile's first key: the
// sort order), or -1 for a dead slot
__device__ __forceinline__ int key_of(const float4& p, const KeyGeo& g)
{
    const int c = __float_as_int(p.w);   // packed i | j << 10 | k << 20
    if (c < 0) return -1;
    const int i = c & 1023, j = (c >> 10) & 1023, k = c >> 20;
    const int ti = i / g.tx, tj = j / g.ty, tk = k / g.tz;
    const int tile = (tk * g.nty + tj) * g.ntx + ti;
    if (g.order == 1) return tile * (g.tx * g.ty * g.tz);
    if (g.order == 2) {
        const int bx = (g.tx + 1) >> 1, by = (g.ty + 1) >> 1;
        return tile * (g.tx * g.ty * g.tz) + (((k - tk * g.tz) >> 1) * by + ((j - tj * g.ty) >> 1)) * bx +
               ((i - ti * g.tx) >> 1);
    }
    return tile * (g.tx * g.ty * g.tz) + ((k - tk * g.tz) * g.ty + (j - tj * g.ty)) * g.tx + (i - ti * g.tx);
}
// FP64: the linear cell index (k*ny + j)*nx + i held in w
__device__ __forceinline__ int key_of(const double4& p, const KeyGeo&) { return p.w < 0.0 ? -1 : (int)p.w; }

// particles per thread and round of the histogram and scatter loops: their
// loads are all issued before the first key's atomic, so one round costs one
// memory latency instead of one per particle
constexpr int kSortUnroll = 4;

template <typename T4>
__global__ void k_hist(const T4* __restrict__ pos, const unsigned long long* nslot, int sp, unsigned int* hist,
                       KeyGeo kg)
{
    const unsigned long long n = nslot[sp];
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    // the loop runs on the warp's first index, so every lane of a warp takes the
    // same rounds (the warp-wide match and shuffle below need all 32)
    for (unsigned long long w0 = blockIdx.x * (unsigned long long)blockDim.x + (threadIdx.x & ~31u); w0 < n;
         w0 += kSortUnroll * stride) {
        const unsigned long long q0 = w0 + (unsigned long long)lane;
        int key[kSortUnroll];
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) {
            const unsigned long long q = q0 + u * stride;
            key[u] = q < n ? key_of(pos[q], kg) : -1;
        }
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) {
            // lanes with the same key (common in nearly sorted input) add once
            const unsigned m = __match_any_sync(0xffffffffu, key[u]);
            if (key[u] >= 0 && lane == __ffs(m) - 1) atomicAdd(hist + key[u], (unsigned int)__popc(m));
        }
    }
}

// exclusive scan of one block of 1024 values; the block total goes to sums[blockIdx]
__global__ void k_scan_block(const unsigned int* in, unsigned int* out, unsigned int* sums, size_t n)
{
    __shared__ unsigned int warp_tot[kScanThreads / 32];
    const size_t base = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * kScanPer;
    unsigned int v[kScanPer];
    unsigned int s = 0;
#pragma unroll
    for (int t = 0; t < kScanPer; ++t) {
        v[t] = (base + t < n) ? in[base + t] : 0u;
        s += v[t];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned int w = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    unsigned int run = (incl - s) + (warp > 0 ? warp_tot[warp - 1] : 0u);
#pragma unroll
    for (int t = 0; t < kScanPer; ++t) {
        if (base + t < n) out[base + t] = run;
        run += v[t];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(unsigned int* out, const unsigned int* offs, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        out[q] += offs[q / kScanBlock];
}

// (mixed precision also lists the new slots of particles in MD cells for the
// next step: md_next / next_n, null for FP64)
template <typename T4>
__global__ void k_scatter(const T4* __restrict__ pos, const T4* __restrict__ vel, const unsigned long long* nslot,
                          int sp, unsigned int* cursor, T4* __restrict__ pos_out, T4* __restrict__ vel_out, KeyGeo kg,
                          int nx, int ny, const int* cell_ng, unsigned int* md_next, unsigned int* next_n)
{
    const unsigned long long n = nslot[sp];
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    // the loop runs on the warp's first index, so every lane of a warp takes the
    // same rounds (the warp-wide match and shuffle below need all 32)
    for (unsigned long long w0 = blockIdx.x * (unsigned long long)blockDim.x + (threadIdx.x & ~31u); w0 < n;
         w0 += kSortUnroll * stride) {
        const unsigned long long q0 = w0 + (unsigned long long)lane;
        T4 p[kSortUnroll], v[kSortUnroll];
        int key[kSortUnroll];
        unsigned int dst[kSortUnroll];
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) {
            const unsigned long long q = q0 + u * stride;
            if (q < n) {
                p[u] = pos[q];
                v[u] = vel[q];
            }
            key[u] = q < n ? key_of(p[u], kg) : -1;
        }
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) {
            // one cursor atomic per group of lanes with the same key; the
            // group's lanes take consecutive slots in lane order
            const unsigned m = __match_any_sync(0xffffffffu, key[u]);
            const int leader = __ffs(m) - 1;
            unsigned int base = 0;
            if (key[u] >= 0 && lane == leader) base = atomicAdd(cursor + key[u], (unsigned int)__popc(m));
            dst[u] = base;
            dst[u] = __shfl_sync(0xffffffffu, dst[u], leader) + (unsigned int)__popc(m & ((1u << lane) - 1u));
        }
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) {
            if (key[u] < 0) continue;
            const unsigned int d = dst[u];
            pos_out[d] = p[u];
            vel_out[d] = v[u];
            if (md_next) {
                const int pc = __float_as_int(p[u].w);   // mixed: packed cell
                if (cell_ng[((pc >> 20) * ny + ((pc >> 10) & 1023)) * nx + (pc & 1023)] != 0)
                    md_next[atomicAdd(next_n, 1u)] = d;
            }
        }
    }
}

// live records (key >= 0) among the slots in use, one add per warp
template <typename T4>
__global__ void k_count_live(const T4* __restrict__ pos, const unsigned long long* nslot, int sp,
                             unsigned long long* live)
{
    const unsigned long long n = nslot[sp];
    const KeyGeo kg{1, 1, 1, 1, 1, 1};
    unsigned int mine = 0;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x)
        mine += key_of(pos[q], kg) >= 0 ? 1u : 0u;
    const unsigned int w = __reduce_add_sync(0xffffffffu, mine);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(live + sp, (unsigned long long)w);
}

__global__ void k_set_nslot(unsigned long long* nslot, int sp, const unsigned int* total)
{
    nslot[sp] = *total;
}

// first slot of every tile after a scatter, which leaves cursor[key] at the end
// of the key's range: tile t starts where key t * per_tile - 1 ends
__global__ void k_tile_ranges(const unsigned int* cursor, unsigned int* tstart, long long ntiles, int per_tile)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t <= ntiles;
         t += (long long)gridDim.x * blockDim.x)
        tstart[t] = t == 0 ? 0u : cursor[t * per_tile - 1];
}

// exclusive scan of n values in place through the per-level scratch buffers
void scan(pic_ctx* c, unsigned int* data, size_t n, int level)
{
    const size_t nb = (n + kScanBlock - 1) / kScanBlock;
    unsigned int* sums = c->scan_tmp[level];
    k_scan_block<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(data, data, sums, n);
    c->launches += 1;
    if (nb > 1) {
        scan(c, sums, nb, level + 1);
        k_scan_add<<<grid_for((int64_t)n, 256, 152 * 8), 256, 0, c->stream>>>(data, sums, n);
        c->launches += 1;
    }
}

}  // namespace

void scan_cells(pic_ctx* c, unsigned int* data) { scan(c, data, c->cells, 0); }

// scratch: one block-sum buffer per scan level, plus a final total slot
// (sized for the sort keys, which are at least as many as the cells)
size_t sort_scratch_setup(pic_ctx* c)
{
    size_t n = std::max(c->nkeys, c->cells);
    size_t bytes = 0;
    c->scan_tmp.clear();
    c->scan_len.clear();
    while (true) {
        const size_t nb = (n + kScanBlock - 1) / kScanBlock;
        unsigned int* p = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (nb + 1));
        if (!p) return 0;
        c->scan_tmp.push_back(p);
        c->scan_len.push_back(nb);
        bytes += sizeof(unsigned int) * (nb + 1);
        if (nb <= 1) break;
        n = nb;
    }
    return bytes + 1;
}

void count_live(pic_ctx* c)
{
    cudaMemsetAsync(c->d_live, 0, 2 * sizeof(unsigned long long), c->stream);
    for (int sp = 0; sp < 2; ++sp) {
        const int grid = grid_for(c->cap[sp], 256, 152 * 8);
        if (c->prec == PIC_MIXED)
            k_count_live<float4><<<grid, 256, 0, c->stream>>>((const float4*)c->pos[sp], c->d_nslot, sp, c->d_live);
        else
            k_count_live<double4><<<grid, 256, 0, c->stream>>>((const double4*)c->pos[sp], c->d_nslot, sp, c->d_live);
    }
    c->launches += 2;
}

void sort_particles(pic_ctx* c, int sp)
{
    const size_t nk = c->nkeys;
    const KeyGeo kg{c->tile[0], c->tile[1], c->tile[2], c->ntile[0], c->ntile[1], c->sort_order};
    cudaMemsetAsync(c->cursor, 0, sizeof(unsigned int) * nk, c->stream);
    const int grid = grid_for(c->cap[sp], 256, 152 * 8);
    if (c->prec == PIC_MIXED)
        k_hist<float4><<<grid, 256, 0, c->stream>>>((const float4*)c->pos[sp], c->d_nslot, sp, c->cursor, kg);
    else
        k_hist<double4><<<grid, 256, 0, c->stream>>>((const double4*)c->pos[sp], c->d_nslot, sp, c->cursor, kg);
    scan(c, c->cursor, nk, 0);
    if (c->prec == PIC_MIXED) cudaMemsetAsync(c->d_lists + 4 + sp, 0, sizeof(unsigned int), c->stream);
    if (c->prec == PIC_MIXED)
        k_scatter<float4><<<grid, 256, 0, c->stream>>>((const float4*)c->pos[sp], (const float4*)c->vel[sp],
                                                       c->d_nslot, sp, c->cursor, (float4*)c->pos_alt[sp],
                                                       (float4*)c->vel_alt[sp], kg, c->nx, c->ny, c->cell_ng,
                                                       c->md_next[sp], c->d_lists + 4 + sp);
    else
        k_scatter<double4><<<grid, 256, 0, c->stream>>>((const double4*)c->pos[sp], (const double4*)c->vel[sp],
                                                        c->d_nslot, sp, c->cursor, (double4*)c->pos_alt[sp],
                                                        (double4*)c->vel_alt[sp], kg, c->nx, c->ny, c->cell_ng,
                                                        (unsigned int*)nullptr, (unsigned int*)nullptr);
    // the last scan level's single block sum is the number of live particles
    k_set_nslot<<<1, 1, 0, c->stream>>>(c->d_nslot, sp, c->scan_tmp.back());
    c->launches += 3;
    if (c->prec == PIC_MIXED) {
        k_tile_ranges<<<grid_for(c->ntiles + 1, 256, 152 * 4), 256, 0, c->stream>>>(
            c->cursor, c->tstart[sp], (long long)c->ntiles, c->tile[0] * c->tile[1] * c->tile[2]);
        c->launches += 1;
    }
    void* t = c->pos[sp]; c->pos[sp] = c->pos_alt[sp]; c->pos_alt[sp] = t;
    t = c->vel[sp]; c->vel[sp] = c->vel_alt[sp]; c->vel_alt[sp] = t;
}

}  // namespace pic

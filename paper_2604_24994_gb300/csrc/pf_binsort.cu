// pf_bin_sort: (cell, tile) instances grouped by tile and sorted per tile by
// (power-distance key, cell index).
//
//   1. per view, the 2D difference grid written by the projection is summed
//      into per-tile instance counts;
//   2. exclusive scans give each tile's bucket start and each (view, cell)
//      its first instance index;
//   3. one thread per instance (load-balanced: big cells do not serialise)
//      finds its cell by binary search, its tile inside the cell's
//      rectangle, and takes a slot in the tile's bucket;
//   4. one CTA per tile sorts the bucket by (key, cell): a bitonic network
//      in shared memory (24 KB for up to 2048 entries, 192 KB for up to
//      16384), or in global memory for larger buckets.
// The result does not depend on the order of the atomic slot grabs: the
// composite key (key, cell) is unique.
#include "pf_internal.cuh"

namespace pf {

constexpr int SCAN_T = 1024;         // threads per scan block
constexpr int SCAN_E = 2 * SCAN_T;   // elements per scan block

// --------------------------------------------------------------- tile counts
__global__ void tile_counts_kernel(const ViewDev *__restrict__ views, int32_t *__restrict__ diff,
                                   uint32_t *__restrict__ tile_cnt) {
    const ViewDev &V = views[blockIdx.x];
    const int gw = V.tiles_x + 1, gh = V.tiles_y + 1;
    int32_t *g = diff + V.diff_base;
    for (int y = threadIdx.x; y < gh; y += blockDim.x) {  // prefix along rows
        int32_t acc = 0;
        for (int x = 0; x < gw; x++) {
            acc += g[y * gw + x];
            g[y * gw + x] = acc;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < gw; x += blockDim.x) {  // then along columns
        int32_t acc = 0;
        for (int y = 0; y < gh; y++) {
            acc += g[y * gw + x];
            g[y * gw + x] = acc;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < V.tiles_x * V.tiles_y; t += blockDim.x) {
        const int y = t / V.tiles_x, x = t - y * V.tiles_x;
        tile_cnt[V.tile_base + t] = (uint32_t)g[y * gw + x];
    }
}

// --------------------------------------------------------- exclusive scans
// Block-local exclusive scan of SCAN_E elements; block sums to `sums`.
__global__ void __launch_bounds__(SCAN_T) scan_blocks_kernel(uint32_t *__restrict__ a, int64_t n,
                                                             uint32_t *__restrict__ sums) {
    __shared__ uint32_t s[SCAN_E];
    const int64_t base = (int64_t)blockIdx.x * SCAN_E;
    const int t = threadIdx.x;
    for (int q = t; q < SCAN_E; q += SCAN_T) s[q] = (base + q < n) ? a[base + q] : 0u;
    __syncthreads();
    // Blelloch up-sweep
    int off = 1;
    for (int d = SCAN_E >> 1; d > 0; d >>= 1) {
        __syncthreads();
        if (t < d) {
            const int ai = off * (2 * t + 1) - 1, bi = off * (2 * t + 2) - 1;
            s[bi] += s[ai];
        }
        off <<= 1;
    }
    __syncthreads();
    if (t == 0) {
        sums[blockIdx.x] = s[SCAN_E - 1];
        s[SCAN_E - 1] = 0;
    }
    for (int d = 1; d < SCAN_E; d <<= 1) {
        off >>= 1;
        __syncthreads();
        if (t < d) {
            const int ai = off * (2 * t + 1) - 1, bi = off * (2 * t + 2) - 1;
            const uint32_t x = s[ai];
            s[ai] = s[bi];
            s[bi] += x;
        }
    }
    __syncthreads();
    for (int q = t; q < SCAN_E; q += SCAN_T)
        if (base + q < n) a[base + q] = s[q];
}

// Exclusive scan of the block sums by one block (any count), total in *total.
__global__ void __launch_bounds__(SCAN_T) scan_sums_kernel(uint32_t *__restrict__ sums, int64_t nb,
                                                           unsigned long long *__restrict__ total,
                                                           unsigned int *__restrict__ overflow,
                                                           unsigned long long cap) {
    __shared__ unsigned long long ws[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += SCAN_T) {
        const int64_t q = base + threadIdx.x;
        unsigned long long x = q < nb ? sums[q] : 0ull;
        unsigned long long incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = ws[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            ws[lane] = w;
        }
        __syncthreads();
        const unsigned long long before = carry + (warp ? ws[warp - 1] : 0ull) + incl - x;
        if (q < nb) sums[q] = (uint32_t)before;
        __syncthreads();
        if (threadIdx.x == SCAN_T - 1) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) {
        *total = carry;
        if (overflow) *overflow = carry > cap ? 1u : 0u;
    }
}

__global__ void __launch_bounds__(SCAN_T) scan_add_kernel(uint32_t *__restrict__ a, int64_t n,
                                                          const uint32_t *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_E;
    const uint32_t add = sums[blockIdx.x];
    for (int q = threadIdx.x; q < SCAN_E; q += SCAN_T)
        if (base + q < n) a[base + q] += add;
}

cudaError_t exclusive_scan(uint32_t *a, int64_t n, uint32_t *tmp, unsigned long long *total,
                           unsigned int *overflow, unsigned long long cap, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + SCAN_E - 1) / SCAN_E;
    scan_blocks_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(a, n, tmp);
    scan_sums_kernel<<<1, SCAN_T, 0, st>>>(tmp, nb, total, overflow, cap);
    scan_add_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(a, n, tmp);
    return cudaGetLastError();
}

// ------------------------------------------------------------- expansion
__device__ __forceinline__ int find_view(const ViewDev *views, int nv, int64_t tile) {
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) expand_kernel(const ViewDev *__restrict__ views, int64_t N, int64_t VN,
                                                     const uint32_t *__restrict__ celloff,
                                                     const ushort4 *__restrict__ rect,
                                                     const unsigned long long *__restrict__ key,
                                                     const uint32_t *__restrict__ tile_start,
                                                     uint32_t *__restrict__ tile_cursor,
                                                     const Counters *__restrict__ ctr, unsigned long long cap,
                                                     unsigned long long *__restrict__ inst_key,
                                                     uint32_t *__restrict__ inst_cell) {
    const unsigned long long total = ctr->total_inst;
    const unsigned long long lim = total < cap ? total : cap;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < lim;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        // last (view, cell) whose first instance is <= k
        int64_t lo = 0, hi = VN - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)celloff[mid] <= k) lo = mid; else hi = mid - 1;
        }
        const int64_t c = lo;
        const int v = (int)(c / N);
        const uint32_t cell = (uint32_t)(c - (int64_t)v * N);
        const ushort4 r = rect[c];
        const uint32_t local = (uint32_t)(k - celloff[c]);
        const uint32_t w = (uint32_t)(r.z - r.x + 1);
        const uint32_t ty = r.y + local / w, tx = r.x + local % w;
        const ViewDev &V = views[v];
        const int64_t tile = V.tile_base + (int64_t)ty * V.tiles_x + tx;
        const uint32_t slot = atomicAdd(&tile_cursor[tile], 1u);
        const unsigned long long pos = (unsigned long long)tile_start[tile] + slot;
        if (pos < cap) {
            inst_key[pos] = key[c];
            inst_cell[pos] = cell;
        }
    }
}

// -------------------------------------------------------------- tile sort
__device__ __forceinline__ bool greater_kc(unsigned long long ka, uint32_t ca, unsigned long long kb, uint32_t cb) {
    return ka > kb || (ka == kb && ca > cb);
}

// Bitonic network in which every comparator puts the minimum at the lower
// index (each merge starts with a "flip" stage), so entries past n behave
// as +infinity and need no storage.
template <typename KeyArr, typename CellArr>
__device__ void bitonic_sort(KeyArr keys, CellArr cells, int n) {
    int P = 1;
    while (P < n) P <<= 1;
    for (int lh = 0; (2 << lh) <= P; lh++) {   // merge blocks of size 2^(lh+1)
        const int half = 1 << lh, size = 2 << lh;
        for (int q = threadIdx.x; q < P / 2; q += blockDim.x) {
            const int blk = (q >> lh) << (lh + 1), r = q & (half - 1);
            const int i = blk + r;
            const int j = blk + size - 1 - r;
            if (j < n) {
                const unsigned long long ki = keys[i], kj = keys[j];
                const uint32_t ci = cells[i], cj = cells[j];
                if (greater_kc(ki, ci, kj, cj)) {
                    keys[i] = kj; keys[j] = ki;
                    cells[i] = cj; cells[j] = ci;
                }
            }
        }
        __syncthreads();
        for (int ls = lh - 1; ls >= 0; ls--) {
            const int stride = 1 << ls;
            for (int q = threadIdx.x; q < P / 2; q += blockDim.x) {
                const int i = ((q >> ls) << (ls + 1)) + (q & (stride - 1));
                const int j = i + stride;
                if (j < n) {
                    const unsigned long long ki = keys[i], kj = keys[j];
                    const uint32_t ci = cells[i], cj = cells[j];
                    if (greater_kc(ki, ci, kj, cj)) {
                        keys[i] = kj; keys[j] = ki;
                        cells[i] = cj; cells[j] = ci;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// One CTA per tile.  Variant <LO, CAP>: buckets with LO < n <= CAP are
// sorted in shared memory; with GLOBAL, buckets above CAP are sorted in
// place in the global scratch arrays.
template <int LO, int CAP, int NT, bool GLOBAL>
__device__ __forceinline__ void sort_tile(int64_t t, const uint32_t *__restrict__ tile_start, unsigned long long cap,
                                          const unsigned long long *inst_key, const uint32_t *inst_cell,
                                          uint32_t *__restrict__ inst_sorted, unsigned long long *tmp_key,
                                          uint32_t *tmp_cell, unsigned long long *sk, uint32_t *sc) {
    unsigned long long s = tile_start[t], e = tile_start[t + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    const int64_t n = (int64_t)(e - s);
    if (n <= LO || n <= 0) return;
    if (n == 1) {
        if (threadIdx.x == 0) inst_sorted[s] = inst_cell[s];
        return;
    }
    if (n <= CAP) {
        for (int q = threadIdx.x; q < n; q += NT) {
            sk[q] = inst_key[s + q];
            sc[q] = inst_cell[s + q];
        }
        __syncthreads();
        bitonic_sort(sk, sc, (int)n);
        for (int q = threadIdx.x; q < n; q += NT) inst_sorted[s + q] = sc[q];
    } else if (GLOBAL) {
        unsigned long long *gk = tmp_key + s;
        uint32_t *gc = tmp_cell + s;
        for (int64_t q = threadIdx.x; q < n; q += NT) {
            gk[q] = inst_key[s + q];
            gc[q] = inst_cell[s + q];
        }
        __syncthreads();
        bitonic_sort(gk, gc, (int)n);
        for (int64_t q = threadIdx.x; q < n; q += NT) inst_sorted[s + q] = gc[q];
    }
}

// One CTA per tile for the lists of at most CAP entries.
template <int CAP, int NT>
__global__ void __launch_bounds__(NT) sort_small_tiles_kernel(const uint32_t *__restrict__ tile_start,
                                                              unsigned long long cap,
                                                              const unsigned long long *inst_key,
                                                              const uint32_t *inst_cell,
                                                              uint32_t *__restrict__ inst_sorted) {
    extern __shared__ unsigned long long sk[];
    uint32_t *sc = reinterpret_cast<uint32_t *>(sk + CAP);
    unsigned long long s = tile_start[blockIdx.x], e = tile_start[blockIdx.x + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    if (e - s > (unsigned long long)CAP) return;  // the persistent kernel sorts it
    sort_tile<0, CAP, NT, false>(blockIdx.x, tile_start, cap, inst_key, inst_cell, inst_sorted, nullptr, nullptr,
                                 sk, sc);
}

// Persistent CTAs over the render order (tiles by decreasing list length,
// bucketed by length / 4): every list longer than LO comes before any list
// shorter than LO, so a CTA stops at the first such list.  Lists up to CAP
// are sorted in shared memory, longer ones in the global scratch arrays.
template <int LO, int CAP, int NT>
__global__ void __launch_bounds__(NT) sort_large_tiles_kernel(const uint32_t *__restrict__ order, int64_t T,
                                                              const uint32_t *__restrict__ tile_start,
                                                              unsigned long long cap,
                                                              const unsigned long long *inst_key,
                                                              const uint32_t *inst_cell,
                                                              uint32_t *__restrict__ inst_sorted,
                                                              unsigned long long *tmp_key, uint32_t *tmp_cell) {
    extern __shared__ unsigned long long sk[];
    uint32_t *sc = reinterpret_cast<uint32_t *>(sk + CAP);
    for (int64_t i = blockIdx.x; i < T; i += gridDim.x) {
        const int64_t t = order[i];
        unsigned long long s = tile_start[t], e = tile_start[t + 1];
        if (s > cap) s = cap;
        if (e > cap) e = cap;
        if (e - s < (unsigned long long)LO) break;  // the same for every thread of the CTA
        sort_tile<LO, CAP, NT, true>(t, tile_start, cap, inst_key, inst_cell, inst_sorted, tmp_key, tmp_cell, sk,
                                     sc);
        __syncthreads();  // shared memory is reused by the next list
    }
}

// Render order: tiles by decreasing list length (bucketed by length / 4),
// so that persistent render CTAs start with the heaviest tiles.
__global__ void __launch_bounds__(1024) tile_order_kernel(const uint32_t *__restrict__ tile_start, int64_t T,
                                                          unsigned long long cap, uint32_t *__restrict__ order) {
    constexpr int NB = 1024;
    __shared__ uint32_t hist[NB];
    for (int b = threadIdx.x; b < NB; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    auto bucket = [&](int64_t t) {
        unsigned long long s = tile_start[t], e = tile_start[t + 1];
        if (s > cap) s = cap;
        if (e > cap) e = cap;
        const unsigned long long c = (e - s) >> 2;
        return NB - 1 - (int)(c < NB - 1 ? c : NB - 1);
    };
    for (int64_t t = threadIdx.x; t < T; t += blockDim.x) atomicAdd(&hist[bucket(t)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {  // 1024 buckets: a serial scan is cheap
        uint32_t acc = 0;
        for (int b = 0; b < NB; b++) {
            const uint32_t x = hist[b];
            hist[b] = acc;
            acc += x;
        }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < T; t += blockDim.x) order[atomicAdd(&hist[bucket(t)], 1u)] = (uint32_t)t;
}

cudaError_t launch_bin_sort(const Plan &p, const WS &w, cudaStream_t st) {
    cudaError_t e;
    const int64_t T = p.total_tiles;
    const int64_t VN = (int64_t)p.n * p.nv;
    e = cudaMemsetAsync(w.counters, 0, sizeof(Counters) - sizeof(((Counters *)0)->stats), st);
    if (e != cudaSuccess) return e;
    // per-tile counts into tile_start[0..T), then exclusive scan over T+1 entries
    e = cudaMemsetAsync(w.tile_start + T, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    tile_counts_kernel<<<p.nv, 256, 0, st>>>(w.views, w.diff, w.tile_start);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = exclusive_scan(w.tile_start, T + 1, w.scan_tmp, nullptr, nullptr, 0, st);
    if (e != cudaSuccess) return e;
    // first instance of every (view, cell); the total decides overflow
    if (VN > 0) {
        e = cudaMemcpyAsync(w.celloff, w.cnt, sizeof(uint32_t) * VN, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        e = exclusive_scan(w.celloff, VN, w.scan_tmp, &w.counters->total_inst, &w.counters->overflow, p.cap, st);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(w.tile_cursor, 0, sizeof(uint32_t) * T, st);
    if (e != cudaSuccess) return e;
    if (VN > 0 && p.cap > 0) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        expand_kernel<<<sms * 8, 256, 0, st>>>(w.views, p.n, VN, w.celloff, w.rect, w.key, w.tile_start,
                                                 w.tile_cursor, w.counters, p.cap, w.inst_key, w.inst_cell);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (T > 0) {
        tile_order_kernel<<<1, 1024, 0, st>>>(w.tile_start, T, p.cap, w.tile_order);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (T > 0) {
        // small buckets (<= 2048) in 24 KB of shared memory, large ones in 192 KB
        constexpr int SMALL = 2048, LARGE = 16384;
        auto ks = sort_small_tiles_kernel<SMALL, 256>;
        auto kl = sort_large_tiles_kernel<SMALL, LARGE, 512>;
        const size_t ss = (size_t)SMALL * 12, sl = (size_t)LARGE * 12;
        cudaFuncSetAttribute(kl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl);
        ks<<<(unsigned)T, 256, ss, st>>>(w.tile_start, p.cap, w.inst_key, w.inst_cell, w.inst_sorted);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        kl<<<(unsigned)(T < sms ? T : sms), 512, sl, st>>>(w.tile_order, T, w.tile_start, p.cap, w.inst_key,
                                                            w.inst_cell, w.inst_sorted, w.sort_tmp_key,
                                                            w.sort_tmp_cell);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pf

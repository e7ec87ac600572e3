// pf_bin_sort: (cell, tile) instances grouped by tile and sorted per tile by
// (power-distance key, cell index).
//
//   1. per view, the 2D difference grid written by the projection is summed
//      into per-tile instance counts;
//   2. exclusive scans give each tile's bucket start and each (view, cell)
//      its first instance index;
//   3. one thread per instance (load-balanced: big cells do not serialise)
//      finds its cell by binary search, its tile inside the cell's
//      rectangle, and takes a slot in the tile's bucket; the tiles are put
//      in render order (longest lists first);
//   4. one CTA per tile sorts the bucket by (key, cell): a bitonic network
//      in 24 KB of shared memory for up to 2048 entries; persistent CTAs,
//      running beside that kernel, a radix sort in 208 KB for up to 16384,
//      and beyond that a split by the leading key bits into runs of at most
//      16384 entries, each sorted in shared memory.
// The result does not depend on the order of the atomic slot grabs: the
// composite key (key, cell) is unique.
#include "pf_internal.cuh"

namespace pf {

constexpr int SCAN_T = 1024;         // threads per scan block
constexpr int SCAN_E = 2 * SCAN_T;   // elements per scan block

// --------------------------------------------------------------- tile counts
// The DIFF_REP copies of the difference grids summed into the first.
__global__ void __launch_bounds__(256) diff_sum_kernel(int32_t *__restrict__ diff, int64_t total) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = 0;
#pragma unroll
        for (int r = 0; r < DIFF_REP; r++) v += diff[total * r + q];
        diff[q] = v;
    }
}

// One CTA per view: the 2D difference grid becomes per-tile counts by an
// inclusive prefix along rows (one warp per row, 32 columns per step, a
// shuffle scan and a carry) and then along columns (one lane per column,
// coalesced row by row).
constexpr int TC_T = 1024;

__global__ void __launch_bounds__(TC_T) tile_counts_kernel(const ViewDev *__restrict__ views, int32_t *__restrict__ diff,
                                                          uint32_t *__restrict__ tile_cnt) {
    const ViewDev &V = views[blockIdx.x];
    const int gw = V.tiles_x + 1, gh = V.tiles_y + 1;
    int32_t *g = diff + V.diff_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int y = warp; y < gh; y += TC_T / 32) {
        int32_t carry = 0;
        for (int x0 = 0; x0 < gw; x0 += 32) {
            const int x = x0 + lane;
            int32_t v = x < gw ? g[y * gw + x] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v += u;
            }
            v += carry;
            if (x < gw) g[y * gw + x] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < gw; x += TC_T) {
        int32_t acc = 0;
        for (int y = 0; y < gh; y++) {
            acc += g[y * gw + x];
            g[y * gw + x] = acc;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < V.tiles_x * V.tiles_y; t += TC_T) {
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

// Instances in chunks of EXP_T * EXP_I consecutive indices per CTA step:
// two threads find the (view, cell) of the chunk's first and last instance
// by binary search over the first-instance offsets in global memory; when
// the cells between them fit, their offsets are staged in shared memory and
// every instance finds its cell there.
constexpr int EXP_T = 256, EXP_I = 4, EXP_CAP = 4096, EXP_NV = 64;

// last c in [lo, hi] with off(c) <= k (off non-decreasing, off(lo) <= k)
template <typename Off>
__device__ __forceinline__ int64_t last_le(Off off, int64_t lo, int64_t hi, unsigned long long k) {
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((unsigned long long)off(mid) <= k) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(EXP_T) expand_kernel(const ViewDev *__restrict__ views, int64_t N, int64_t VN,
                                                       const uint32_t *__restrict__ celloff,
                                                       const ushort4 *__restrict__ rect,
                                                       const unsigned long long *__restrict__ key,
                                                       const uint32_t *__restrict__ tile_start,
                                                       uint32_t *__restrict__ tile_cursor,
                                                       const Counters *__restrict__ ctr, unsigned long long cap,
                                                       unsigned long long *__restrict__ inst_key,
                                                       uint32_t *__restrict__ inst_cell) {
    __shared__ uint32_t soff[EXP_CAP];
    __shared__ int64_t range[2];
    // each view's first tile and tiles per row (of the first EXP_NV views)
    __shared__ int64_t vtb[EXP_NV];
    __shared__ int32_t vtx[EXP_NV];
    const int nv = (int)(VN / N);
    for (int q = threadIdx.x; q < nv && q < EXP_NV; q += EXP_T) {
        vtb[q] = views[q].tile_base;
        vtx[q] = views[q].tiles_x;
    }
    __syncthreads();
    const unsigned long long total = ctr->total_inst;
    const unsigned long long lim = total < cap ? total : cap;
    constexpr unsigned long long CH = (unsigned long long)EXP_T * EXP_I;
    auto goff = [&](int64_t c) { return celloff[c]; };
    for (unsigned long long k0 = (unsigned long long)blockIdx.x * CH; k0 < lim;
         k0 += (unsigned long long)gridDim.x * CH) {
        const unsigned long long k1 = (k0 + CH < lim ? k0 + CH : lim) - 1;
        if (threadIdx.x == 0) range[0] = last_le(goff, 0, VN - 1, k0);
        if (threadIdx.x == 32) range[1] = last_le(goff, 0, VN - 1, k1);
        __syncthreads();
        const int64_t lo = range[0], hi = range[1];
        const bool staged = hi - lo + 1 <= EXP_CAP;
        if (staged)
            for (int64_t q = threadIdx.x; q <= hi - lo; q += EXP_T) soff[q] = celloff[lo + q];
        __syncthreads();
        for (int r = 0; r < EXP_I; r++) {
            const unsigned long long k = k0 + (unsigned long long)r * EXP_T + threadIdx.x;
            if (k > k1) break;
            const int64_t c = staged ? last_le([&](int64_t x) { return soff[x - lo]; }, lo, hi, k)
                                     : last_le(goff, lo, hi, k);
            const int v = (int)(c / N);
            const uint32_t cell = (uint32_t)(c - (int64_t)v * N);
            const ushort4 rc = rect[c];
            const uint32_t local = (uint32_t)(k - celloff[c]);
            const uint32_t w = (uint32_t)(rc.z - rc.x + 1);
            const uint32_t ty = rc.y + local / w, tx = rc.x + local % w;
            const int64_t tile = v < EXP_NV ? vtb[v] + (int64_t)ty * vtx[v] + tx
                                            : views[v].tile_base + (int64_t)ty * views[v].tiles_x + tx;
            const uint32_t slot = atomicAdd(&tile_cursor[tile], 1u);
            const unsigned long long pos = (unsigned long long)tile_start[tile] + slot;
            if (pos < cap) {
                inst_key[pos] = key[c];
                inst_cell[pos] = cell;
            }
        }
        __syncthreads();  // soff and range are rewritten for the next chunk
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

// One stable counting pass over a 4-bit digit: entries move from ia to ib,
// dig(x) is entry x's digit.
template <int NT, typename Dig>
__device__ __forceinline__ void radix_pass(int b, int e, const uint16_t *ia, uint16_t *ib, uint16_t *cnt,
                                           unsigned long long *red, Dig dig) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // this thread's digit counts, eight bits each (E <= 32)
    unsigned long long c0 = 0ull, c1 = 0ull;
    for (int i = b; i < e; i++) {
        const unsigned dg = dig(ia[i]);
        if (dg < 8)
            c0 += 1ull << (8 * dg);
        else
            c1 += 1ull << (8 * (dg - 8));
    }
#pragma unroll
    for (int dg = 0; dg < 16; dg++)
        cnt[dg * NT + t] = (uint16_t)(((dg < 8 ? c0 >> (8 * dg) : c1 >> (8 * (dg - 8)))) & 0xffull);
    __syncthreads();
    // exclusive scan of cnt in (digit, thread) order: 16 entries per thread
    uint16_t *mine = cnt + 16 * t;
    unsigned run = 0;
#pragma unroll
    for (int r = 0; r < 16; r++) run += mine[r];
    unsigned incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    unsigned before = incl - run;
    for (int w = 0; w < warp; w++) before += (unsigned)red[w];
#pragma unroll
    for (int r = 0; r < 16; r++) {
        const unsigned x = mine[r];
        mine[r] = (uint16_t)before;
        before += x;
    }
    __syncthreads();
    for (int i = b; i < e; i++) {
        const uint16_t x = ia[i];
        const unsigned dg = dig(x);
        const unsigned pos = cnt[dg * NT + t];
        cnt[dg * NT + t] = (uint16_t)(pos + 1u);
        ib[pos] = x;
    }
    __syncthreads();
}

// OR ^ AND of v over the CTA: the bits in which the values differ.
template <int NT>
__device__ __forceinline__ unsigned long long varying_bits(unsigned long long o, unsigned long long a,
                                                           unsigned long long *red) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, d);
        a &= __shfl_xor_sync(0xffffffffu, a, d);
    }
    if (lane == 0) {
        red[warp] = o;
        red[NW + warp] = a;
    }
    __syncthreads();
    unsigned long long vo = 0ull, va = ~0ull;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        vo |= red[w];
        va &= red[NW + w];
    }
    __syncthreads();  // red is reused by the scans
    return vo ^ va;
}

// Lists whose equal keys form more than this many adjacent pairs are sorted
// again with the cell index as the low-order part of the key (the insertion
// fix-up below is quadratic in a run's length).
constexpr int TIE_INSERT_MAX = 64;

// The rare path of radix_sort_tile: the list sorted again from bucket order,
// the cell index's varying digits first and then the key's, so that equal
// keys end in cell order.  Out of line: it keeps the common path's registers.
template <int NT>
static __device__ __noinline__ uint16_t *radix_resort_with_cells(int n, const uint32_t *__restrict__ cells,
                                                                 const unsigned long long *keys, uint16_t *ia,
                                                                 uint16_t *ib, uint16_t *cnt,
                                                                 unsigned long long *red,
                                                                 unsigned long long vary) {
    const int t = threadIdx.x;
    const int E = (n + NT - 1) / NT;
    const int b = min(n, t * E), e = min(n, b + E);
    unsigned long long co = 0ull, ca = ~0ull;
    for (int q = t; q < n; q += NT) {
        ia[q] = (uint16_t)q;
        co |= cells[q];
        ca &= cells[q];
    }
    const unsigned long long cvary = varying_bits<NT>(co, ca, red);
    for (int sh = 0; sh < 32; sh += 4) {
        if (((cvary >> sh) & 15ull) == 0ull) continue;
        radix_pass<NT>(b, e, ia, ib, cnt, red, [cells, sh](uint16_t x) { return (cells[x] >> sh) & 15u; });
        uint16_t *sw = ia;
        ia = ib;
        ib = sw;
    }
    for (int sh = 0; sh < 64; sh += 4) {
        if (((vary >> sh) & 15ull) == 0ull) continue;
        radix_pass<NT>(b, e, ia, ib, cnt, red, [keys, sh](uint16_t x) { return (unsigned)(keys[x] >> sh) & 15u; });
        uint16_t *sw = ia;
        ia = ib;
        ib = sw;
    }
    return ia;
}

// Stable LSD radix sort of one tile's list in shared memory, 4-bit digits.
// The 64-bit keys stay in place (keys[q] = key of bucket entry q); 16-bit
// entry indices move between ia and ib.  Thread t owns the contiguous
// entries [t E, (t + 1) E), E = ceil(n / NT) <= 32, so the order of equal
// digits is (thread, position) order, the list order before the pass.
// Digit positions where every key has the same bits are skipped.  Equal
// keys end in bucket order, which the atomic slot grabs made arbitrary: a
// final pass puts each run of equal keys in cell order (by insertion when
// they are few, else by sorting again with the cell index's digits first).
// gkey / cells: the bucket in global memory; keys: n words, ia / ib: n entries, cnt:
// 16 NT counters, red: 2 NT / 32 words of shared memory.  Returns the
// array (ia or ib) that holds the sorted entry order.
template <int NT>
__device__ uint16_t *radix_sort_tile(int n, const unsigned long long *__restrict__ gkey,
                                     const uint32_t *__restrict__ cells, unsigned long long *keys, uint16_t *ia,
                                     uint16_t *ib, uint16_t *cnt, unsigned long long *red) {
    const int t = threadIdx.x;
    unsigned long long o = 0ull, a = ~0ull;
    for (int q = t; q < n; q += NT) {
        const unsigned long long k = gkey[q];
        keys[q] = k;
        o |= k;
        a &= k;
        ia[q] = (uint16_t)q;
    }
    const unsigned long long vary = varying_bits<NT>(o, a, red);
    const int E = (n + NT - 1) / NT;
    const int b = min(n, t * E), e = min(n, b + E);
    for (int sh = 0; sh < 64; sh += 4) {
        if (((vary >> sh) & 15ull) == 0ull) continue;  // the same for every thread
        radix_pass<NT>(b, e, ia, ib, cnt, red, [keys, sh](uint16_t x) { return (unsigned)(keys[x] >> sh) & 15u; });
        uint16_t *sw = ia;
        ia = ib;
        ib = sw;
    }
    // equal keys end in bucket order; put them in cell order
    int mine = 0;
    for (int q = t; q + 1 < n; q += NT) mine += keys[ia[q]] == keys[ia[q + 1]];
    if (!__syncthreads_or(mine > 0)) return ia;
    unsigned long long *tot = red;  // the CTA's count of adjacent equal pairs
    if (t == 0) *tot = 0ull;
    __syncthreads();
    if (mine) atomicAdd(tot, (unsigned long long)mine);
    __syncthreads();
    const int nties = (int)*tot;
    __syncthreads();
    if (nties > TIE_INSERT_MAX) return radix_resort_with_cells<NT>(n, cells, keys, ia, ib, cnt, red, vary);
    // few ties: each run of equal keys into cell order (insertion sort by its first thread)
    for (int q = t; q + 1 < n; q += NT) {
        const unsigned long long k = keys[ia[q]];
        if (k != keys[ia[q + 1]] || (q > 0 && keys[ia[q - 1]] == k)) continue;
        int r = q + 2;
        while (r < n && keys[ia[r]] == k) r++;
        for (int i = q + 1; i < r; i++) {
            const uint16_t x = ia[i];
            const uint32_t cx = cells[x];
            int j = i - 1;
            while (j >= q && cells[ia[j]] > cx) {
                ia[j + 1] = ia[j];
                j--;
            }
            ia[j + 1] = x;
        }
    }
    __syncthreads();
    return ia;
}

// Shared memory of a sorting CTA: keys [CAP] (8 B), two entry-index arrays
// [CAP] (2 B each; the bitonic path keeps cells [CAP] (4 B) there), digit
// counters [16 NT] (2 B), reduction words [2 NT / 32] (8 B).
template <int CAP, int NT>
struct SortSmem {
    static constexpr size_t keys = 0, ia = keys + (size_t)CAP * 8, ib = ia + (size_t)CAP * 2,
                            cnt = ib + (size_t)CAP * 2, red = cnt + (size_t)16 * NT * 2,
                            bytes = red + (size_t)2 * (NT / 32) * 8;
};

// Lists of at most this many entries take the bitonic network, longer ones
// the radix sort (measured on GB300: the 256 thread CTA sorts lists of up
// to 2048 entries faster with the network, the 512 thread CTA lists of
// 2049-16384 entries three times faster with the radix sort).
constexpr int BITONIC_MAX = 2048;

// A list of 2 <= m <= CAP entries in global memory (keys gk, cells gc),
// sorted in shared memory by (key, cell); its cells in order to out.
template <int CAP, int NT>
__device__ void sort_run_shared(int m, const unsigned long long *gk, const uint32_t *gc, uint32_t *out,
                                char *smem) {
    using L = SortSmem<CAP, NT>;
    unsigned long long *sk = reinterpret_cast<unsigned long long *>(smem + L::keys);
    if (m <= BITONIC_MAX) {
        uint32_t *sc = reinterpret_cast<uint32_t *>(smem + L::ia);
        for (int q = threadIdx.x; q < m; q += NT) {
            sk[q] = gk[q];
            sc[q] = gc[q];
        }
        __syncthreads();
        bitonic_sort(sk, sc, m);
        for (int q = threadIdx.x; q < m; q += NT) out[q] = sc[q];
    } else if constexpr (CAP > BITONIC_MAX) {
        const uint16_t *ord = radix_sort_tile<NT>(
            m, gk, gc, sk, reinterpret_cast<uint16_t *>(smem + L::ia), reinterpret_cast<uint16_t *>(smem + L::ib),
            reinterpret_cast<uint16_t *>(smem + L::cnt), reinterpret_cast<unsigned long long *>(smem + L::red));
        for (int q = threadIdx.x; q < m; q += NT) out[q] = gc[ord[q]];
    }
    __syncthreads();  // shared memory is reused by the next list
}

// ------------------------------------------------ lists above CAP entries
// A list too long for shared memory is split by the 8 most significant bits
// in which its keys differ: a counting pass, then every entry moves to its
// bucket in the other pair of global arrays (same offsets; the order within
// a bucket does not matter).  The buckets partition the key range in order,
// so runs of consecutive buckets holding at most CAP entries in all are
// each sorted in shared memory as one list, completely by (key, cell), and
// the runs end to end are the sorted list.  A bucket above CAP is split
// again by the next 8 bits (at most 8 levels: each consumes 8 key bits); one
// whose keys are all equal, or that finds the stack full, is sorted in place
// in global memory by the bitonic network.
constexpr int BIG_DIG = 8, BIG_NB = 1 << BIG_DIG, BIG_STACK = 128;

struct BigSeg {
    uint32_t off, m;  // first entry (from the list's start) and length
    int buf, depth;   // where its entries are (0: instance arrays, 1: scratch arrays); splits above it
};
struct BigRun {
    uint32_t start, m;  // first entry (from the segment's start) and length
    int global, pad;    // 1: one bucket above CAP, sorted in global memory
};

// Shared memory after SortSmem: bucket counts and cursors, the runs of the
// current split, the stack of buckets still to split, two counters.
struct BigSmem {
    static constexpr size_t hist = 0, cur = hist + BIG_NB * 4, run = cur + BIG_NB * 4,
                            stk = run + (BIG_NB + 1) * sizeof(BigRun), ctl = stk + BIG_STACK * sizeof(BigSeg),
                            bytes = ctl + 16;
};

template <int CAP, int NT>
static __device__ __forceinline__ void sort_long_list(uint32_t n, unsigned long long *k0, uint32_t *c0,
                                                   unsigned long long *k1, uint32_t *c1, uint32_t *out,
                                                   char *smem) {
    using L = SortSmem<CAP, NT>;
    char *xs = smem + L::bytes;
    uint32_t *hist = reinterpret_cast<uint32_t *>(xs + BigSmem::hist);
    uint32_t *cur = reinterpret_cast<uint32_t *>(xs + BigSmem::cur);
    BigRun *run = reinterpret_cast<BigRun *>(xs + BigSmem::run);
    BigSeg *stk = reinterpret_cast<BigSeg *>(xs + BigSmem::stk);
    int *ctl = reinterpret_cast<int *>(xs + BigSmem::ctl);
    unsigned long long *red = reinterpret_cast<unsigned long long *>(smem + L::red);
    const int t = threadIdx.x, lane = t & 31;
    const uint32_t w0 = (uint32_t)(t & ~31);  // this warp's first entry of each round
    if (t == 0) stk[0] = BigSeg{0u, n, 0, 0};
    int sp = 1;  // the same in every thread
    for (int guard = 0; sp > 0 && guard < (1 << 20); guard++) {
        __syncthreads();  // the stack written by thread 0 is visible
        const BigSeg g = stk[--sp];
        unsigned long long *sk = (g.buf ? k1 : k0) + g.off, *dk = (g.buf ? k0 : k1) + g.off;
        uint32_t *sc = (g.buf ? c1 : c0) + g.off, *dc = (g.buf ? c0 : c1) + g.off;
        uint32_t *o = out + g.off;
        unsigned long long vo = 0ull, va = ~0ull;
        for (uint32_t q = t; q < g.m; q += NT) {
            const unsigned long long k = sk[q];
            vo |= k;
            va &= k;
        }
        const unsigned long long vary = varying_bits<NT>(vo, va, red);  // also: every thread has read g
        if (vary == 0ull || g.depth >= 8) {  // all keys equal: the cells decide
            bitonic_sort(sk, sc, (int)g.m);
            for (uint32_t q = t; q < g.m; q += NT) o[q] = sc[q];
            continue;
        }
        const int hb = 63 - __clzll((long long)vary);
        const int sh = hb >= BIG_DIG - 1 ? hb - (BIG_DIG - 1) : 0;
        for (int d = t; d < BIG_NB; d += NT) hist[d] = 0u;
        __syncthreads();
        // counts: rounds of 32 consecutive entries per warp, one atomic per digit and round
        for (uint32_t q0 = w0; q0 < g.m; q0 += NT) {
            const uint32_t q = q0 + lane;
            const unsigned d = q < g.m ? (unsigned)(sk[q] >> sh) & (BIG_NB - 1) : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&hist[d], (unsigned)__popc(peers));
        }
        __syncthreads();
        if (t == 0) {  // bucket offsets, the runs, and the buckets to split again
            uint32_t acc = 0u, rs = 0u, rm = 0u;
            int nr = 0;
            for (int d = 0; d < BIG_NB; d++) {
                const uint32_t c = hist[d];
                cur[d] = acc;
                if (c > (uint32_t)CAP) {
                    if (rm) run[nr++] = BigRun{rs, rm, 0, 0};
                    rm = 0u;
                    if (sp < BIG_STACK)
                        stk[sp++] = BigSeg{g.off + acc, c, g.buf ^ 1, g.depth + 1};
                    else
                        run[nr++] = BigRun{acc, c, 1, 0};
                } else if (c) {
                    if (rm + c > (uint32_t)CAP) {
                        run[nr++] = BigRun{rs, rm, 0, 0};
                        rm = 0u;
                    }
                    if (!rm) rs = acc;
                    rm += c;
                }
                acc += c;
            }
            if (rm) run[nr++] = BigRun{rs, rm, 0, 0};
            ctl[0] = nr;
            ctl[1] = sp;
        }
        __syncthreads();
        const int nr = ctl[0];
        sp = ctl[1];
        // every entry to its bucket: a rank among the round's equal digits after the bucket's cursor
        for (uint32_t q0 = w0; q0 < g.m; q0 += NT) {
            const uint32_t q = q0 + lane;
            const bool ok = q < g.m;
            const unsigned long long k = ok ? sk[q] : 0ull;
            const uint32_t c = ok ? sc[q] : 0u;
            const unsigned d = ok ? (unsigned)(k >> sh) & (BIG_NB - 1) : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0u;
            if (ok && lane == leader) base = atomicAdd(&cur[d], (unsigned)__popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (ok) {
                const uint32_t pos = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
                dk[pos] = k;
                dc[pos] = c;
            }
        }
        __syncthreads();  // the moved entries are visible to the CTA
        for (int r = 0; r < nr; r++) {
            const BigRun R = run[r];
            if (R.global) {
                bitonic_sort(dk + R.start, dc + R.start, (int)R.m);
                for (uint32_t q = t; q < R.m; q += NT) o[R.start + q] = dc[R.start + q];
            } else if (R.m == 1u) {
                if (t == 0) o[R.start] = dc[R.start];
            } else {
                sort_run_shared<CAP, NT>((int)R.m, dk + R.start, dc + R.start, o + R.start, smem);
            }
        }
    }
}

// One CTA per tile.  Variant <LO, CAP>: buckets with LO < n <= CAP are
// sorted in shared memory; with GLOBAL, buckets above CAP by splitting
// them (sort_long_list), with the global scratch arrays beside the
// instance arrays.
template <int LO, int CAP, int NT, bool GLOBAL>
__device__ __forceinline__ void sort_tile(int64_t t, const uint32_t *__restrict__ tile_start, unsigned long long cap,
                                          const unsigned long long *inst_key, const uint32_t *inst_cell,
                                          uint32_t *__restrict__ inst_sorted, unsigned long long *tmp_key,
                                          uint32_t *tmp_cell, char *smem) {
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
        sort_run_shared<CAP, NT>((int)n, inst_key + s, inst_cell + s, inst_sorted + s, smem);
    } else if constexpr (GLOBAL) {
        // the instance arrays are scratch once the lists are sorted: the
        // splits move entries between them and the scratch arrays
        sort_long_list<CAP, NT>((uint32_t)n, const_cast<unsigned long long *>(inst_key) + s,
                                const_cast<uint32_t *>(inst_cell) + s, tmp_key + s, tmp_cell + s, inst_sorted + s,
                                smem);
    }
}

// One CTA per tile for the lists of at most CAP entries, CTAs in the render
// order (longest lists first, so that the last wave holds the short ones).
// Launched as a programmatic dependent of the long-list kernel, so the two
// run side by side (each touches only its own tiles' ranges of the
// instance, scratch and sorted arrays); the last CTA
// waits for that kernel's completion before it exits, so this kernel's
// completion, which the next launch on the stream waits for, implies both.
template <int CAP, int NT>
__global__ void __launch_bounds__(NT) sort_small_tiles_kernel(const uint32_t *__restrict__ order,
                                                              const uint32_t *__restrict__ tile_start,
                                                              unsigned long long cap,
                                                              const unsigned long long *inst_key,
                                                              const uint32_t *inst_cell,
                                                              uint32_t *__restrict__ inst_sorted) {
    extern __shared__ unsigned long long smem_sort[];
    const int64_t tt = order[blockIdx.x];
    unsigned long long s = tile_start[tt], e = tile_start[tt + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    if (e - s <= (unsigned long long)CAP)  // longer lists: the persistent kernel sorts them
        sort_tile<0, CAP, NT, false>(tt, tile_start, cap, inst_key, inst_cell, inst_sorted, nullptr, nullptr,
                                     reinterpret_cast<char *>(smem_sort));
    if (blockIdx.x == gridDim.x - 1) asm volatile("griddepcontrol.wait;" ::: "memory");
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
    extern __shared__ unsigned long long smem_sort[];
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");  // the short-list sort may start now
    for (int64_t i = blockIdx.x; i < T; i += gridDim.x) {
        const int64_t t = order[i];
        unsigned long long s = tile_start[t], e = tile_start[t + 1];
        if (s > cap) s = cap;
        if (e > cap) e = cap;
        if (e - s < (unsigned long long)LO) break;  // the same for every thread of the CTA
        sort_tile<LO, CAP, NT, true>(t, tile_start, cap, inst_key, inst_cell, inst_sorted, tmp_key, tmp_cell,
                                     reinterpret_cast<char *>(smem_sort));
        __syncthreads();  // shared memory is reused by the next list
    }
}

// Render order: tiles by decreasing list length (bucketed by length / 4),
// so that persistent render CTAs start with the heaviest tiles.  One CTA of
// 1024 threads, one per length bucket.
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
    {  // exclusive scan of the 1024 buckets, one per thread: warp scans, then a scan of the warp sums
        __shared__ uint32_t wsum[NB / 32];
        const int b = threadIdx.x, lane = b & 31;
        const uint32_t x = hist[b];
        uint32_t v = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) wsum[b >> 5] = v;
        __syncthreads();
        if (b < NB / 32) {
            uint32_t u = wsum[b];
            for (int o = 1; o < NB / 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, u, o);
                if (lane >= o) u += y;
            }
            wsum[b] = u;
        }
        __syncthreads();
        hist[b] = v - x + ((b >> 5) ? wsum[(b >> 5) - 1] : 0u);
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
    if (p.total_diff > 0) {
        const int64_t nb = (p.total_diff + 255) / 256;
        diff_sum_kernel<<<(unsigned)(nb < 1024 ? nb : 1024), 256, 0, st>>>(w.diff, p.total_diff);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    tile_counts_kernel<<<p.nv, TC_T, 0, st>>>(w.views, w.diff, w.tile_start);
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
        expand_kernel<<<sms * 8, EXP_T, 0, st>>>(w.views, p.n, VN, w.celloff, w.rect, w.key, w.tile_start,
                                                 w.tile_cursor, w.counters, p.cap, w.inst_key, w.inst_cell);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (T > 0) {
        tile_order_kernel<<<1, 1024, 0, st>>>(w.tile_start, T, p.cap, w.tile_order);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (T > 0) {
        // small buckets (<= 2048) in 24 KB of shared memory (bitonic), large ones in 208 KB (radix;
        // above 16384 entries split by their leading key bits first, with 8 KB more)
        constexpr int SMALL = 2048, LARGE = 16384;
        auto ks = sort_small_tiles_kernel<SMALL, 256>;
        auto kl = sort_large_tiles_kernel<SMALL, LARGE, 512>;
        static_assert(SMALL <= BITONIC_MAX, "the small-list kernel sorts with the bitonic network only");
        const size_t ss = (size_t)SMALL * 12, sl = SortSmem<LARGE, 512>::bytes + BigSmem::bytes;
        cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
        cudaFuncSetAttribute(kl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl);
        // the long lists first (a few persistent CTAs, one per SM), the short
        // ones beside them on the SMs that the first kernel leaves free
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        kl<<<(unsigned)(T < sms ? T : sms), 512, sl, st>>>(w.tile_order, T, w.tile_start, p.cap, w.inst_key,
                                                            w.inst_cell, w.inst_sorted, w.sort_tmp_key,
                                                            w.sort_tmp_cell);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.gridDim = dim3((unsigned)T);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = ss;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, ks, (const uint32_t *)w.tile_order, (const uint32_t *)w.tile_start, p.cap,
                               (const unsigned long long *)w.inst_key, (const uint32_t *)w.inst_cell, w.inst_sorted);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pf

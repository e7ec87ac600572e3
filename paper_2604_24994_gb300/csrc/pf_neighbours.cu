// Neighbour lists on the GPU: for every cell i, the K sites j whose radical
// planes (Sec. 3.2, Eq. power bisector) lie nearest p_i, ranked by the signed
// distance of the plane from p_i,
//
//     t_ij = (|p_j - p_i|^2 + w_i - w_j) / (2 |p_j - p_i|),
//
// ties by j, and the bound radius clipped to R_i <= t_(K+1) so that no site
// missing from the list can cut the cell's sphere.  This is the step the paper
// does with GPU collision detection over the bounding spheres (Sec. 3.3, the
// Cech graph); with R_i clipped, a fixed-width list is exact for any K.
//
// Structure (one stream, no host synchronisation, no allocation):
//   1. bounding box of the sites (atomics on order-preserving float bits);
//   2. 30-bit Morton codes over the box, stable LSD radix sort (4 x 8 bits);
//   3. binary radix tree over the sorted codes (Karras 2012: the split of a
//      node's range is its highest differing key bit, ties broken by index);
//   4. bottom-up refit: each internal node gets the box of its sites and
//      their largest weight;
//   5. one thread per site (in Morton order) keeps the K+1 smallest (t, j):
//      it seeds the list with its neighbours in Morton order, then walks the
//      tree, skipping every subtree whose lower bound on t exceeds the
//      current (K+1)-th value.  Over a box at distance D with largest weight
//      W, t >= min over L >= D of (L^2 + w_i - W) / (2L), which is
//      (D^2 + w_i - W) / (2D) when w_i - W <= D^2 and sqrt(w_i - W)
//      otherwise.  Bounds and screens run in float with a margin well above
//      their rounding error; every t that can enter the list is computed in
//      FP64 with explicitly rounded operations (no contraction), so the
//      ranking, the ties and the clipped radius are exact functions of the
//      float inputs.
#include <algorithm>

#include "pf_internal.cuh"

namespace pf {

cudaError_t exclusive_scan(uint32_t *a, int64_t n, uint32_t *tmp, unsigned long long *total,
                           unsigned int *overflow, unsigned long long cap, cudaStream_t st);

namespace {

constexpr int NB_T = 256;                  // threads per block (sort, build)
constexpr int NB_ITEMS = 16;               // keys per thread per radix block
constexpr int NB_CHUNK = NB_T * NB_ITEMS;  // keys per radix block
constexpr int NB_QT = 64;                  // threads per query block
constexpr int NB_STACK = 64;               // tree depth is at most 30 + 32 key bits
constexpr float NB_MARGIN = 0x1p-18f;      // screen / bound margin, relative
constexpr int NB_EXTRA = 16;               // band-set entries beyond the K+1
constexpr int NB_BUCKET = 8;               // nodes over at most this many sites are scanned

struct NbParams {
    unsigned int lo[3], hi[3];  // order-preserving bits of the bounding box
    unsigned int clipped;       // cells whose R was clipped
    unsigned int stack_overflow;
};

struct NbLayout {
    uint64_t params, code0, val0, code1, val1, hist, scan_tmp, parent, child, rng, box, flag, site, redo, total;
    int64_t nblk, hist_n;
};

NbLayout nb_layout(int64_t n) {
    NbLayout L{};
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    const int64_t nn = n > 0 ? n : 1;
    L.nblk = (nn + NB_CHUNK - 1) / NB_CHUNK;
    L.hist_n = 256 * L.nblk;
    L.params = take(sizeof(NbParams));
    L.code0 = take(4 * (uint64_t)nn);
    L.val0 = take(4 * (uint64_t)nn);
    L.code1 = take(4 * (uint64_t)nn);
    L.val1 = take(4 * (uint64_t)nn);
    L.hist = take(4 * (uint64_t)L.hist_n);
    L.scan_tmp = take(4 * (uint64_t)((L.hist_n + 2047) / 2048 + 1));
    L.parent = take(4 * (uint64_t)(2 * nn));
    L.child = take(4 * (uint64_t)(2 * nn));
    L.rng = take(8 * (uint64_t)nn);
    L.box = take(32 * (uint64_t)(2 * nn));
    L.flag = take(4 * (uint64_t)nn);
    L.site = take(16 * (uint64_t)nn);
    L.redo = take((uint64_t)nn);
    L.total = o;
    return L;
}

__device__ __forceinline__ unsigned int f2o(float f) {  // order-preserving float bits
    const unsigned int b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float o2f(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void nb_init_kernel(NbParams *P) {
    for (int a = 0; a < 3; a++) {
        P->lo[a] = 0xffffffffu;
        P->hi[a] = 0u;
    }
    P->clipped = 0;
    P->stack_overflow = 0;
}

__global__ void __launch_bounds__(NB_T) nb_bbox_kernel(const float *__restrict__ pos, int64_t n,
                                                       NbParams *__restrict__ P) {
    unsigned int lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; a++) {
            const unsigned int u = f2o(pos[3 * i + a]);
            lo[a] = min(lo[a], u);
            hi[a] = max(hi[a], u);
        }
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&P->lo[a], lo[a]);
            atomicMax(&P->hi[a], hi[a]);
        }
    }
}

__device__ __forceinline__ unsigned int spread10(unsigned int x) {  // 10 bits -> every third bit
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void __launch_bounds__(NB_T) nb_morton_kernel(const float *__restrict__ pos, int64_t n,
                                                         const NbParams *__restrict__ P,
                                                         uint32_t *__restrict__ code, uint32_t *__restrict__ val) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned int c = 0;
    for (int a = 0; a < 3; a++) {
        const float lo = o2f(P->lo[a]), hi = o2f(P->hi[a]);
        const float ext = hi - lo;
        // NaN or a zero extent map to 0 (fmaxf drops NaN)
        float u = ext > 0.0f ? (pos[3 * i + a] - lo) / ext : 0.0f;
        u = fminf(fmaxf(u * 1024.0f, 0.0f), 1023.0f);
        c |= spread10((unsigned int)u) << (2 - a);
    }
    code[i] = c;
    val[i] = (uint32_t)i;
}

// ----------------------------------------------------- stable LSD radix sort
__global__ void __launch_bounds__(NB_T) nb_hist_kernel(const uint32_t *__restrict__ code, int64_t n, int shift,
                                                       uint32_t *__restrict__ hist, int64_t nblk) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = blockIdx.x * (int64_t)NB_CHUNK;
    for (int r = 0; r < NB_ITEMS; r++) {
        const int64_t i = base + r * NB_T + threadIdx.x;
        if (i < n) atomicAdd(&h[(code[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// hist holds, digit-major, the exclusive scan of the block histograms: the
// first output slot of (digit, block).  Keys keep their input order within a
// digit: rounds of 256 in index order, warps in order, lanes in order.
__global__ void __launch_bounds__(NB_T) nb_scatter_kernel(const uint32_t *__restrict__ code_in,
                                                          const uint32_t *__restrict__ val_in, int64_t n, int shift,
                                                          const uint32_t *__restrict__ hist, int64_t nblk,
                                                          uint32_t *__restrict__ code_out,
                                                          uint32_t *__restrict__ val_out) {
    constexpr int NW = NB_T / 32;
    __shared__ unsigned int run[256];
    __shared__ unsigned int wc[NW][256];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    run[t] = hist[t * nblk + blockIdx.x];
    for (int q = 0; q < NW; q++) wc[q][t] = 0;
    __syncthreads();
    const int64_t base = blockIdx.x * (int64_t)NB_CHUNK;
    for (int r = 0; r < NB_ITEMS; r++) {
        const int64_t i = base + r * NB_T + t;
        const bool valid = i < n;
        const uint32_t c = valid ? code_in[i] : 0u, v = valid ? val_in[i] : 0u;
        const unsigned int d = valid ? ((c >> shift) & 255u) : 256u;
        const unsigned int peers = __match_any_sync(0xffffffffu, d);
        const unsigned int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned int off = run[d] + rank;
            for (int q = 0; q < warp; q++) off += wc[q][d];
            code_out[off] = c;
            val_out[off] = v;
        }
        __syncthreads();
        unsigned int tot = 0;
        for (int q = 0; q < NW; q++) {
            tot += wc[q][t];
            wc[q][t] = 0;
        }
        run[t] += tot;
        __syncthreads();
    }
}

// ------------------------------------------------------- binary radix tree
// Node ids: internal nodes 0 .. n-2 (root 0), leaf s (sorted position) is
// n - 1 + s.
__device__ __forceinline__ int nb_delta(const uint32_t *__restrict__ code, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = code[i], b = code[j];
    return a != b ? __clz(a ^ b) : 32 + __clz((unsigned int)(i ^ j));
}

__global__ void __launch_bounds__(NB_T) nb_tree_kernel(const uint32_t *__restrict__ code, int64_t n,
                                                       int32_t *__restrict__ child, int32_t *__restrict__ parent,
                                                       int2 *__restrict__ rng) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = nb_delta(code, n, i, i + 1) - nb_delta(code, n, i, i - 1) >= 0 ? 1 : -1;
    const int dmin = nb_delta(code, n, i, i - d);
    int64_t lmax = 2;
    while (nb_delta(code, n, i, i + lmax * d) > dmin) lmax *= 2;
    int64_t l = 0;
    for (int64_t s = lmax / 2; s >= 1; s /= 2)
        if (nb_delta(code, n, i, i + (l + s) * d) > dmin) l += s;
    const int64_t j = i + l * d;
    const int dnode = nb_delta(code, n, i, j);
    int64_t s = 0, step = l;
    do {
        step = (step + 1) >> 1;
        if (nb_delta(code, n, i, i + (s + step) * d) > dnode) s += step;
    } while (step > 1);
    const int64_t g = i + s * d + min(d, 0);
    const int64_t left = min(i, j) == g ? (n - 1 + g) : g;
    const int64_t right = max(i, j) == g + 1 ? (n - 1 + g + 1) : g + 1;
    rng[i] = make_int2((int)min(i, j), (int)max(i, j));  // the sorted positions under node i
    child[2 * i] = (int32_t)left;
    child[2 * i + 1] = (int32_t)right;
    parent[left] = (int32_t)i;
    parent[right] = (int32_t)i;
    if (i == 0) parent[0] = -1;
}

// Leaves write their site (sorted copy and point box), then each thread walks
// up; the second child to arrive at a node forms its box.
__global__ void __launch_bounds__(NB_T) nb_refit_kernel(const float *__restrict__ pos, const float *__restrict__ w,
                                                        const uint32_t *__restrict__ val, int64_t n,
                                                        const int32_t *__restrict__ child,
                                                        const int32_t *__restrict__ parent,
                                                        float4 *__restrict__ box, unsigned int *__restrict__ flag,
                                                        float4 *__restrict__ site, NbParams *__restrict__ P) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t i = val[s];
    const float4 p = make_float4(pos[3 * (int64_t)i], pos[3 * (int64_t)i + 1], pos[3 * (int64_t)i + 2], w[i]);
    site[s] = p;
    const int64_t leaf = n - 1 + s;
    box[2 * leaf] = p;
    box[2 * leaf + 1] = make_float4(p.x, p.y, p.z, 0.0f);
    if (n < 2) return;
    int64_t node = parent[leaf];
    for (int up = 0; node >= 0; up++) {
        if (up >= 2 * NB_STACK) {  // deeper than any radix tree over 62-bit keys
            atomicOr(&P->stack_overflow, 1u);
            return;
        }
        __threadfence();
        if (atomicAdd(&flag[node], 1u) == 0u) return;  // the sibling subtree is not done yet
        const int64_t a = child[2 * node], b = child[2 * node + 1];
        const float4 alo = __ldcg(&box[2 * a]), ahi = __ldcg(&box[2 * a + 1]);
        const float4 blo = __ldcg(&box[2 * b]), bhi = __ldcg(&box[2 * b + 1]);
        box[2 * node] = make_float4(fminf(alo.x, blo.x), fminf(alo.y, blo.y), fminf(alo.z, blo.z), fmaxf(alo.w, blo.w));
        box[2 * node + 1] = make_float4(fmaxf(ahi.x, bhi.x), fmaxf(ahi.y, bhi.y), fmaxf(ahi.z, bhi.z), 0.0f);
        node = parent[node];
    }
}

// ------------------------------------------------------------------ queries
// t_ij in FP64, each operation rounded as written (the oracle evaluates the
// same expression in the same order)
__device__ __forceinline__ double plane_t64(float4 pi, float4 pj) {
    const double dx = __dsub_rn((double)pj.x, (double)pi.x);
    const double dy = __dsub_rn((double)pj.y, (double)pi.y);
    const double dz = __dsub_rn((double)pj.z, (double)pi.z);
    const double L2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (!(L2 > 0.0)) return CUDART_INF;  // coincident sites: no plane
    const double L = __dsqrt_rn(L2);
    return __ddiv_rn(__dsub_rn(__dadd_rn(L2, (double)pi.w), (double)pj.w), __dmul_rn(2.0, L));
}

// Hardware approximations (a few ulp, flush to zero): the screens below
// carry a margin of 2^-18, far above their error.
__device__ __forceinline__ float nb_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float nb_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// t_ij in float and an interval [lb, ub] that holds the FP64 value: the
// margin is 2^-18 of the terms' magnitudes, well above the float rounding
// of the few operations involved.  (-inf, +inf) where float cannot tell.
__device__ __forceinline__ float2 plane_band(float4 pi, float4 pj) {
    const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
    const float L2 = dx * dx + dy * dy + dz * dz;
    if (L2 > 0x1p-100f) {  // well inside the normal range: the approximations hold
        const float inv2L = 0.5f * nb_rcp(nb_sqrt(L2));
        const float tf = (L2 + pi.w - pj.w) * inv2L;
        const float M = NB_MARGIN * ((L2 + fabsf(pi.w) + fabsf(pj.w)) * inv2L + fabsf(tf));
        const float lb = tf - M, ub = tf + M;
        if (lb <= ub) return make_float2(lb, ub);  // false for NaN
    }
    return make_float2(-CUDART_INF_F, CUDART_INF_F);
}

// Exact set: the K+1 smallest (t, j) so far in FP64, ascending, in shared
// memory (entry e of a thread at [e * NB_QT]: threads side by side).
struct NbExact {
    double *t;
    int32_t *j;
    int m, cap;
    __device__ __forceinline__ double limit() const { return m == cap ? t[(cap - 1) * NB_QT] : CUDART_INF; }
    __device__ __forceinline__ bool visit(float4 pi, float4 pj, uint32_t jj, int64_t) {
        const float2 bd = plane_band(pi, pj);
        if ((double)bd.x > limit()) return true;
        const double tt = plane_t64(pi, pj);
        if (!(tt < CUDART_INF)) return true;  // +inf or NaN: no plane
        if (m == cap) {
            const double tl = t[(cap - 1) * NB_QT];
            if (!(tt < tl || (tt == tl && (int32_t)jj < j[(cap - 1) * NB_QT]))) return true;
        }
        int q = m < cap ? m++ : cap - 1;
        while (q > 0) {
            const double tp = t[(q - 1) * NB_QT];
            const int32_t jp = j[(q - 1) * NB_QT];
            if (!(tp > tt || (tp == tt && jp > (int32_t)jj))) break;
            t[q * NB_QT] = tp;
            j[q * NB_QT] = jp;
            q--;
        }
        t[q * NB_QT] = tt;
        j[q * NB_QT] = (int32_t)jj;
        return true;
    }
};

// Band set: every candidate that may still be among the K+1 smallest, kept
// as float intervals sorted by upper end.  U, the (K+1)-th smallest upper
// end, bounds t_(K+1) from above; a site whose lower end exceeds U can never
// enter.  Entries hold the sorted position q (the site's j is looked up at
// the end).  visit() returns false when the set is full of candidates that
// cannot be told apart in float (the caller then redoes the cell exactly).
struct NbBand {
    float2 *b;
    int32_t *q;
    int m, kk, cap;
    __device__ __forceinline__ float U() const { return m >= kk ? b[(kk - 1) * NB_QT].y : CUDART_INF_F; }
    __device__ __forceinline__ double limit() const { return (double)U(); }
    __device__ __forceinline__ bool visit(float4 pi, float4 pj, uint32_t, int64_t qq) {
        const float2 bd = plane_band(pi, pj);
        if (bd.x > U()) return true;
        if (m == cap) {  // drop the entries beyond the first K+1 that can no longer enter
            const float Uc = U();
            int w = kk;
            for (int e = kk; e < m; e++) {
                const float2 x = b[e * NB_QT];
                if (!(x.x > Uc)) {
                    b[w * NB_QT] = x;
                    q[w * NB_QT] = q[e * NB_QT];
                    w++;
                }
            }
            m = w;
            if (m == cap) return false;
        }
        int p = m++;
        while (p > 0) {
            const float2 x = b[(p - 1) * NB_QT];
            if (!(x.y > bd.y)) break;
            b[p * NB_QT] = x;
            q[p * NB_QT] = q[(p - 1) * NB_QT];
            p--;
        }
        b[p * NB_QT] = bd;
        q[p * NB_QT] = (int32_t)qq;
        const float Un = U();
        while (m > kk && b[(m - 1) * NB_QT].x > Un) m--;
        return true;
    }
};

// Lower bound on t_ij over the sites of a node box (lo.w = their largest w).
__device__ __forceinline__ float nb_bound(float4 pi, float4 lo, float4 hi) {
    const float ax = fmaxf(fmaxf(lo.x - pi.x, pi.x - hi.x), 0.0f);
    const float ay = fmaxf(fmaxf(lo.y - pi.y, pi.y - hi.y), 0.0f);
    const float az = fmaxf(fmaxf(lo.z - pi.z, pi.z - hi.z), 0.0f);
    const float D2 = ax * ax + ay * ay + az * az;
    const float c = pi.w - lo.w;
    if (c > D2) return c > 0x1p-100f ? nb_sqrt(c) * (1.0f - 4.0f * NB_MARGIN) : 0.0f;
    if (!(D2 > 0x1p-100f)) return -CUDART_INF_F;
    const float inv2D = 0.5f * nb_rcp(nb_sqrt(D2));
    const float b = (D2 + c) * inv2D;
    return b - NB_MARGIN * ((D2 + fabsf(pi.w) + fabsf(lo.w)) * inv2D + fabsf(b));
}

// Offer site i (sorted position s) its candidates: about K+2 neighbours in
// Morton order, then every site of the tree not ruled out by a node bound
// (nodes over at most NB_BUCKET sites are scanned site by site).  False if
// the set overflowed.
template <class Set>
__device__ __forceinline__ bool nb_walk(Set &set, const float4 *__restrict__ site, const uint32_t *__restrict__ val,
                                        int64_t n, int k, int64_t s, float4 pi, const int32_t *__restrict__ child,
                                        const int2 *__restrict__ rng, const float4 *__restrict__ box,
                                        NbParams *__restrict__ P) {
    const int64_t h = (k + 2) / 2 + 1;
    const int64_t q0 = s - h > 0 ? s - h : 0, q1 = s + h < n - 1 ? s + h : n - 1;
    for (int64_t q = q0; q <= q1; q++)
        if (q != s && !set.visit(pi, site[q], val[q], q)) return false;
    if (n < 2) return true;
    int32_t stack[NB_STACK];
    int sp = 0;
    stack[sp++] = 0;
    for (int64_t pops = 0; sp > 0; pops++) {
        if (pops >= n) {  // a tree has n - 1 internal nodes, each taken at most once
            atomicOr(&P->stack_overflow, 1u);
            return true;
        }
        const int64_t node = stack[--sp];
        const int64_t c2[2] = {child[2 * node], child[2 * node + 1]};
        bool keep[2] = {false, false};
        float key[2] = {0.0f, 0.0f};
        for (int e = 0; e < 2; e++) {
            const int64_t c = c2[e];
            int64_t lo_q, hi_q;
            if (c >= n - 1) {  // one site
                lo_q = hi_q = c - (n - 1);
            } else {
                const float b = nb_bound(pi, box[2 * c], box[2 * c + 1]);
                if ((double)b > set.limit()) continue;  // NaN admits the node
                const int2 r = rng[c];
                if (r.y - r.x >= NB_BUCKET) {
                    keep[e] = true;
                    key[e] = b == b ? b : -CUDART_INF_F;
                    continue;
                }
                lo_q = r.x;
                hi_q = r.y;
            }
            for (int64_t q = lo_q; q <= hi_q; q++)
                if ((q < q0 || q > q1) && !set.visit(pi, site[q], val[q], q)) return false;
        }
        // push the farther child first so the nearer one is taken next
        const int first = (keep[0] && keep[1] && key[0] <= key[1]) ? 1 : 0;
        for (int e = 0; e < 2; e++) {
            const int x = e == 0 ? first : 1 - first;
            if (!keep[x]) continue;
            if (sp < NB_STACK) {
                stack[sp++] = (int32_t)c2[x];
            } else {
                atomicOr(&P->stack_overflow, 1u);
            }
        }
    }
    return true;
}

// Write cell i's list from its first min(m, k) ascending entries (finite t)
// and clip R by the (K+1)-th value.
__device__ __forceinline__ void nb_emit(const double *t, const int32_t *j, int m, int k, uint32_t i,
                                        const float *__restrict__ R_in, int32_t *__restrict__ nbr,
                                        float *__restrict__ R_out, NbParams *__restrict__ P) {
    for (int q = 0; q < k; q++)
        nbr[(int64_t)i * k + q] = (q < m && t[q * NB_QT] < CUDART_INF) ? j[q * NB_QT] : -1;
    const double tk1 = k < m ? t[k * NB_QT] : CUDART_INF;
    const float Ri = R_in[i];
    if (tk1 < (double)Ri) {
        R_out[i] = __double2float_rd(fmax(tk1, 0.0));
        atomicAdd(&P->clipped, 1u);
    } else {
        R_out[i] = Ri;
    }
}

// Main query: the band set, then FP64 values for its
// survivors only, sorted by (t, j).  Cells whose set overflowed are marked
// in `redo` for nb_exact_kernel.
__global__ void __launch_bounds__(NB_QT) nb_query_kernel(const float4 *__restrict__ site,
                                                         const uint32_t *__restrict__ val, int64_t n, int k,
                                                         int extra, const int32_t *__restrict__ child,
                                                         const int2 *__restrict__ rng,
                                                         const float4 *__restrict__ box,
                                                         const float *__restrict__ R_in, int32_t *__restrict__ nbr,
                                                         float *__restrict__ R_out, uint8_t *__restrict__ redo,
                                                         NbParams *__restrict__ P) {
    extern __shared__ __align__(16) unsigned char nb_smem[];
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t i = val[s];
    const float4 pi = site[s];
    NbBand set;
    set.kk = k + 1;
    set.cap = k + 1 + extra;
    set.b = (float2 *)nb_smem + threadIdx.x;
    set.q = (int32_t *)((float2 *)nb_smem + set.cap * NB_QT) + threadIdx.x;
    set.m = 0;
    if (!nb_walk(set, site, val, n, k, s, pi, child, rng, box, P)) {
        redo[s] = 1;
        return;
    }
    // exact values in place of the intervals (same 8 bytes), j in place of q
    double *t = (double *)set.b;
    int32_t *j = set.q;
    for (int e = 0; e < set.m; e++) {
        const int64_t q = j[e * NB_QT];
        t[e * NB_QT] = plane_t64(pi, site[q]);
        j[e * NB_QT] = (int32_t)val[q];
    }
    // nearly sorted already: insertion sort by (t, j); +inf (no plane) last
    for (int e = 1; e < set.m; e++) {
        const double te = t[e * NB_QT];
        const int32_t je = j[e * NB_QT];
        int p = e;
        while (p > 0) {
            const double tp = t[(p - 1) * NB_QT];
            const int32_t jp = j[(p - 1) * NB_QT];
            if (!(tp > te || (tp == te && jp > je))) break;
            t[p * NB_QT] = tp;
            j[p * NB_QT] = jp;
            p--;
        }
        t[p * NB_QT] = te;
        j[p * NB_QT] = je;
    }
    nb_emit(t, j, set.m, k, i, R_in, nbr, R_out, P);
}

// Fallback for the cells marked in `redo`: the same walk with an exact FP64
// list (every value that can enter is computed on the spot).
__global__ void __launch_bounds__(NB_QT) nb_exact_kernel(const float4 *__restrict__ site,
                                                         const uint32_t *__restrict__ val, int64_t n, int k,
                                                         const int32_t *__restrict__ child,
                                                         const int2 *__restrict__ rng,
                                                         const float4 *__restrict__ box,
                                                         const float *__restrict__ R_in, int32_t *__restrict__ nbr,
                                                         float *__restrict__ R_out,
                                                         const uint8_t *__restrict__ redo,
                                                         NbParams *__restrict__ P) {
    extern __shared__ __align__(16) unsigned char nb_smem[];
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n || !redo[s]) return;
    const uint32_t i = val[s];
    const float4 pi = site[s];
    NbExact set;
    set.cap = k + 1;
    set.t = (double *)nb_smem + threadIdx.x;
    set.j = (int32_t *)((double *)nb_smem + set.cap * NB_QT) + threadIdx.x;
    set.m = 0;
    nb_walk(set, site, val, n, k, s, pi, child, rng, box, P);
    nb_emit(set.t, set.j, set.m, k, i, R_in, nbr, R_out, P);
}

// ------------------------------------------- Cech adjacency: L_connect
// The connectivity loss of Sec. 4 / appendix sums over the Cech adjacency
// of the bounding spheres: every j whose sphere overlaps cell i's.  The same
// Morton-ordered radix tree, refit with the spheres' boxes, answers "which
// spheres overlap sphere i" for every i; the pairs found are the exact
// adjacency (the box test is conservative), and each cell gathers its own
// loss and gradient (no atomics: the pair (i, j) is met from both sides).

// Leaves: the site and radius (sorted copy) and the sphere's box, rounded
// outwards; internal nodes: the union of their children's boxes.
__global__ void __launch_bounds__(NB_T) cc_refit_kernel(const float *__restrict__ pos, const float *__restrict__ R,
                                                        const uint32_t *__restrict__ val, int64_t n,
                                                        const int32_t *__restrict__ child,
                                                        const int32_t *__restrict__ parent,
                                                        float4 *__restrict__ box, unsigned int *__restrict__ flag,
                                                        float4 *__restrict__ site, NbParams *__restrict__ P) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t i = val[s];
    const float r = fmaxf(R[i], 0.0f);
    const float4 p = make_float4(pos[3 * (int64_t)i], pos[3 * (int64_t)i + 1], pos[3 * (int64_t)i + 2], r);
    site[s] = p;
    const int64_t leaf = n - 1 + s;
    box[2 * leaf] = make_float4(__fsub_rd(p.x, r), __fsub_rd(p.y, r), __fsub_rd(p.z, r), 0.0f);
    box[2 * leaf + 1] = make_float4(__fadd_ru(p.x, r), __fadd_ru(p.y, r), __fadd_ru(p.z, r), 0.0f);
    if (n < 2) return;
    int64_t node = parent[leaf];
    for (int up = 0; node >= 0; up++) {
        if (up >= 2 * NB_STACK) {
            atomicOr(&P->stack_overflow, 1u);
            return;
        }
        __threadfence();
        if (atomicAdd(&flag[node], 1u) == 0u) return;  // the sibling subtree is not done yet
        const int64_t a = child[2 * node], b = child[2 * node + 1];
        const float4 alo = __ldcg(&box[2 * a]), ahi = __ldcg(&box[2 * a + 1]);
        const float4 blo = __ldcg(&box[2 * b]), bhi = __ldcg(&box[2 * b + 1]);
        box[2 * node] = make_float4(fminf(alo.x, blo.x), fminf(alo.y, blo.y), fminf(alo.z, blo.z), 0.0f);
        box[2 * node + 1] = make_float4(fmaxf(ahi.x, bhi.x), fmaxf(ahi.y, bhi.y), fmaxf(ahi.z, bhi.z), 0.0f);
        node = parent[node];
    }
}

// Can sphere (pi.xyz, pi.w) meet the box?  Conservative: the squared
// distance from the centre to the box against R^2 with a relative margin
// far above the float rounding of these few operations (NaN admits).
__device__ __forceinline__ bool cc_box_hit(float4 pi, float4 lo, float4 hi) {
    const float ax = fmaxf(fmaxf(lo.x - pi.x, pi.x - hi.x), 0.0f);
    const float ay = fmaxf(fmaxf(lo.y - pi.y, pi.y - hi.y), 0.0f);
    const float az = fmaxf(fmaxf(lo.z - pi.z, pi.z - hi.z), 0.0f);
    const float D2 = ax * ax + ay * ay + az * az;
    return !(D2 > pi.w * pi.w * (1.0f + 1e-5f) + 1e-30f);
}

// One pair in FP64 from the float inputs: o = R_i + R_j - |p_j - p_i|; if
// o > 0 the loss gets o^2, and the gradient of the loss summed over cells
// (where the pair appears twice, in L(i) and in L(j)) gets 4 o for R_i and
// 4 o (p_j - p_i) / d for p_i (no direction when the sites coincide).
struct CcAcc {
    double loss = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, gr = 0.0;
    unsigned int pairs = 0;
    __device__ __forceinline__ void pair(float4 pi, float4 pj) {
        // float screen first: pairs farther apart than R_i + R_j by more than
        // the screen's rounding (far below its 1e-5 relative margin) add nothing
        const float fx = pj.x - pi.x, fy = pj.y - pi.y, fz = pj.z - pi.z, rs = pi.w + pj.w;
        if (fx * fx + fy * fy + fz * fz > rs * rs * (1.0f + 1e-5f) + 1e-30f) return;
        const double dx = (double)pj.x - (double)pi.x, dy = (double)pj.y - (double)pi.y,
                     dz = (double)pj.z - (double)pi.z;
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        const double o = ((double)pi.w + (double)pj.w) - d;
        if (!(o > 0.0)) return;
        pairs++;
        loss += o * o;
        gr += 4.0 * o;
        if (d > 0.0) {
            const double f = 4.0 * o / d;
            gx += f * dx;
            gy += f * dy;
            gz += f * dz;
        }
    }
};

__global__ void __launch_bounds__(NB_QT) cc_query_kernel(const float4 *__restrict__ site,
                                                         const uint32_t *__restrict__ val, int64_t n,
                                                         const int32_t *__restrict__ child,
                                                         const int2 *__restrict__ rng,
                                                         const float4 *__restrict__ box, float *__restrict__ loss,
                                                         float *__restrict__ gpos, float *__restrict__ gR,
                                                         NbParams *__restrict__ P) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t i = val[s];
    const float4 pi = site[s];
    CcAcc acc;
    if (n >= 2) {
        int32_t stack[NB_STACK];
        int sp = 0;
        stack[sp++] = 0;
        for (int64_t pops = 0; sp > 0; pops++) {
            if (pops >= n) {  // a tree has n - 1 internal nodes, each taken at most once
                atomicOr(&P->stack_overflow, 1u);
                break;
            }
            const int64_t node = stack[--sp];
            for (int e = 0; e < 2; e++) {
                const int64_t c = child[2 * node + e];
                if (!cc_box_hit(pi, box[2 * c], box[2 * c + 1])) continue;
                int64_t lo_q, hi_q;
                if (c >= n - 1) {  // one site
                    lo_q = hi_q = c - (n - 1);
                } else {
                    const int2 r = rng[c];
                    if (r.y - r.x >= NB_BUCKET) {
                        if (sp < NB_STACK) stack[sp++] = (int32_t)c;
                        else atomicOr(&P->stack_overflow, 1u);
                        continue;
                    }
                    lo_q = r.x;
                    hi_q = r.y;
                }
                for (int64_t q = lo_q; q <= hi_q; q++)
                    if (q != s) acc.pair(pi, site[q]);
            }
        }
    }
    loss[i] = (float)acc.loss;
    if (gpos) {
        gpos[3 * (int64_t)i] += (float)acc.gx;
        gpos[3 * (int64_t)i + 1] += (float)acc.gy;
        gpos[3 * (int64_t)i + 2] += (float)acc.gz;
        gR[i] += (float)acc.gr;
    }
}

__global__ void nb_finish_kernel(const NbParams *__restrict__ P, uint32_t *__restrict__ n_clipped,
                                 uint32_t *__restrict__ status) {
    if (n_clipped) *n_clipped = P->clipped;
    if (status) *status = P->stack_overflow;
}

// Steps 1-3 of the build, shared by the neighbour lists and the Cech
// query: bounding box, Morton codes, stable radix sort (the sorted codes and
// site ids end in code0 / val0), the radix tree, and the refit's arrival
// flags and parent links reset.
static cudaError_t nb_sort_and_tree(const float *pos, int64_t n, const NbLayout &L, char *b, cudaStream_t st) {
    NbParams *P = (NbParams *)(b + L.params);
    uint32_t *code0 = (uint32_t *)(b + L.code0), *val0 = (uint32_t *)(b + L.val0);
    uint32_t *code1 = (uint32_t *)(b + L.code1), *val1 = (uint32_t *)(b + L.val1);
    uint32_t *hist = (uint32_t *)(b + L.hist), *scan_tmp = (uint32_t *)(b + L.scan_tmp);
    int32_t *parent = (int32_t *)(b + L.parent), *child = (int32_t *)(b + L.child);
    int2 *rng = (int2 *)(b + L.rng);
    unsigned int *flag = (unsigned int *)(b + L.flag);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid_n = (unsigned)((n + NB_T - 1) / NB_T);
    nb_init_kernel<<<1, 1, 0, st>>>(P);
    cudaError_t e = cudaMemsetAsync(flag, 0, 4 * (size_t)n, st);
    if (!e) e = cudaMemsetAsync(parent, 0xff, 4 * (size_t)(2 * n), st);  // -1: the refit walk stops there
    if (e) return e;
    const unsigned grid_bb = (unsigned)std::min<int64_t>((int64_t)2 * sms, (int64_t)grid_n);
    nb_bbox_kernel<<<grid_bb, NB_T, 0, st>>>(pos, n, P);
    nb_morton_kernel<<<grid_n, NB_T, 0, st>>>(pos, n, P, code0, val0);
    uint32_t *ci = code0, *vi = val0, *co = code1, *vo = val1;
    for (int shift = 0; shift < 32; shift += 8) {
        nb_hist_kernel<<<(unsigned)L.nblk, NB_T, 0, st>>>(ci, n, shift, hist, L.nblk);
        e = exclusive_scan(hist, L.hist_n, scan_tmp, nullptr, nullptr, 0, st);
        if (e) return e;
        nb_scatter_kernel<<<(unsigned)L.nblk, NB_T, 0, st>>>(ci, vi, n, shift, hist, L.nblk, co, vo);
        uint32_t *tc = ci, *tv = vi;
        ci = co;
        vi = vo;
        co = tc;
        vo = tv;
    }
    // four passes: the sorted keys are back in code0 / val0
    if (n >= 2) nb_tree_kernel<<<(unsigned)((n - 1 + NB_T - 1) / NB_T), NB_T, 0, st>>>(code0, n, child, parent, rng);
    return cudaGetLastError();
}

}  // namespace
}  // namespace pf

using namespace pf;

extern "C" uint64_t pf_neighbours_workspace_bytes(int32_t n_cells) {
    return n_cells < 0 ? 0 : nb_layout(n_cells).total;
}

extern "C" pf_status pf_build_neighbours(const float *pos, const float *w, const float *R_in, int32_t n_cells,
                                         int32_t k_nbr, int32_t *nbr, float *R_out, uint32_t *n_clipped,
                                         uint32_t *status, void *ws, uint64_t ws_bytes, void *stream) {
    set_error("%s", "");
    if (n_cells < 0 || n_cells > PF_NEIGHBOURS_MAX_CELLS || k_nbr < 0 || k_nbr > MAX_K) {
        set_error("pf_build_neighbours: %d cells / %d neighbours outside [0, %d] / [0, %d]", n_cells, k_nbr,
                  PF_NEIGHBOURS_MAX_CELLS, MAX_K);
        return PF_ERR_INVALID_ARG;
    }
    const int64_t n = n_cells;
    if (n > 0 && (!pos || !w || !R_in || !R_out || (k_nbr > 0 && !nbr) || !ws)) {
        set_error("pf_build_neighbours: null pointer");
        return PF_ERR_INVALID_ARG;
    }
    const NbLayout L = nb_layout(n);
    if (n > 0 && ws_bytes < L.total) {
        set_error("pf_build_neighbours: workspace %llu bytes < %llu", (unsigned long long)ws_bytes,
                  (unsigned long long)L.total);
        return PF_ERR_CAPACITY;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        cudaError_t e = cudaSuccess;
        if (n_clipped) e = cudaMemsetAsync(n_clipped, 0, sizeof(uint32_t), st);
        if (!e && status) e = cudaMemsetAsync(status, 0, sizeof(uint32_t), st);
        return cuda_status(e, "pf_build_neighbours");
    }
    char *b = (char *)ws;
    NbParams *P = (NbParams *)(b + L.params);
    uint32_t *val0 = (uint32_t *)(b + L.val0);
    int32_t *parent = (int32_t *)(b + L.parent), *child = (int32_t *)(b + L.child);
    int2 *rng = (int2 *)(b + L.rng);
    float4 *box = (float4 *)(b + L.box), *site = (float4 *)(b + L.site);
    unsigned int *flag = (unsigned int *)(b + L.flag);

    cudaError_t e = nb_sort_and_tree(pos, n, L, b, st);
    if (e) return cuda_status(e, "pf_build_neighbours: tree");
    const unsigned grid_n = (unsigned)((n + NB_T - 1) / NB_T);
    nb_refit_kernel<<<grid_n, NB_T, 0, st>>>(pos, w, val0, n, child, parent, box, flag, site, P);
    uint8_t *redo = (uint8_t *)(b + L.redo);
    e = cudaMemsetAsync(redo, 0, (size_t)n, st);
    if (e) return cuda_status(e, "pf_build_neighbours: memset");
    const unsigned grid_q = (unsigned)((n + NB_QT - 1) / NB_QT);
    const size_t smem_band = (size_t)(k_nbr + 1 + NB_EXTRA) * NB_QT * (sizeof(float2) + sizeof(int32_t));
    e = cudaFuncSetAttribute(nb_query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_band);
    if (e) return cuda_status(e, "pf_build_neighbours: shared memory");
    nb_query_kernel<<<grid_q, NB_QT, smem_band, st>>>(site, val0, n, k_nbr, NB_EXTRA, child, rng, box, R_in, nbr,
                                                     R_out, redo, P);
    const size_t smem_exact = (size_t)(k_nbr + 1) * NB_QT * (sizeof(double) + sizeof(int32_t));
    e = cudaFuncSetAttribute(nb_exact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_exact);
    if (e) return cuda_status(e, "pf_build_neighbours: shared memory");
    nb_exact_kernel<<<grid_q, NB_QT, smem_exact, st>>>(site, val0, n, k_nbr, child, rng, box, R_in, nbr, R_out, redo,
                                                       P);
    if (n_clipped || status) nb_finish_kernel<<<1, 1, 0, st>>>(P, n_clipped, status);
    return cuda_status(cudaGetLastError(), "pf_build_neighbours");
}

extern "C" uint64_t pf_connect_cech_workspace_bytes(int32_t n_cells) {
    return n_cells < 0 ? 0 : nb_layout(n_cells).total;
}

extern "C" pf_status pf_connect_cech(const float *pos, const float *R, int32_t n_cells, float *loss,
                                     float *grad_pos, float *grad_R, uint32_t *status, void *ws, uint64_t ws_bytes,
                                     void *stream) {
    set_error("%s", "");
    if (n_cells < 0 || n_cells > PF_NEIGHBOURS_MAX_CELLS) {
        set_error("pf_connect_cech: %d cells outside [0, %d]", n_cells, PF_NEIGHBOURS_MAX_CELLS);
        return PF_ERR_INVALID_ARG;
    }
    if ((grad_pos == nullptr) != (grad_R == nullptr)) {
        set_error("pf_connect_cech: grad_pos and grad_R are given together or not at all");
        return PF_ERR_INVALID_ARG;
    }
    const int64_t n = n_cells;
    if (n > 0 && (!pos || !R || !loss || !ws)) {
        set_error("pf_connect_cech: null pointer");
        return PF_ERR_INVALID_ARG;
    }
    const NbLayout L = nb_layout(n);
    if (n > 0 && ws_bytes < L.total) {
        set_error("pf_connect_cech: workspace %llu bytes < %llu", (unsigned long long)ws_bytes,
                  (unsigned long long)L.total);
        return PF_ERR_CAPACITY;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        cudaError_t e = status ? cudaMemsetAsync(status, 0, sizeof(uint32_t), st) : cudaSuccess;
        return cuda_status(e, "pf_connect_cech");
    }
    char *b = (char *)ws;
    NbParams *P = (NbParams *)(b + L.params);
    uint32_t *val0 = (uint32_t *)(b + L.val0);
    int32_t *parent = (int32_t *)(b + L.parent), *child = (int32_t *)(b + L.child);
    int2 *rng = (int2 *)(b + L.rng);
    float4 *box = (float4 *)(b + L.box), *site = (float4 *)(b + L.site);
    unsigned int *flag = (unsigned int *)(b + L.flag);
    cudaError_t e = nb_sort_and_tree(pos, n, L, b, st);
    if (e) return cuda_status(e, "pf_connect_cech: tree");
    const unsigned grid_n = (unsigned)((n + NB_T - 1) / NB_T);
    cc_refit_kernel<<<grid_n, NB_T, 0, st>>>(pos, R, val0, n, child, parent, box, flag, site, P);
    cc_query_kernel<<<(unsigned)((n + NB_QT - 1) / NB_QT), NB_QT, 0, st>>>(site, val0, n, child, rng, box, loss,
                                                                           grad_pos, grad_R, P);
    if (status) nb_finish_kernel<<<1, 1, 0, st>>>(P, nullptr, status);
    return cuda_status(cudaGetLastError(), "pf_connect_cech");
}

// sort.cu -- device-wide exclusive scan and stable LSD radix sort of
// (u32 key, u32 value) pairs.  Both read their element count from device
// memory so that a whole frame can be enqueued (and graph-captured) without
// a host round trip; grids are sized by capacity and idle blocks exit.
#include "gsr_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ u32 warp_incl_scan(u32 v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u32 t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// inclusive scan over a block of NT threads; returns inclusive value, total in *tot
template <int NT>
__device__ __forceinline__ u32 block_incl_scan(u32 v, u32 *tot)
{
    __shared__ u32 warp_tot[NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    u32 inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        u32 t = lane < NT / 32 ? warp_tot[lane] : 0u;
        t = warp_incl_scan(t);
        if (lane < NT / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    u32 before = w > 0 ? warp_tot[w - 1] : 0u;
    *tot = warp_tot[NT / 32 - 1];
    __syncthreads();
    return inc + before;
}

__device__ __forceinline__ int64_t eff_n(int64_t n_cap, const u32 *d_n)
{
    if (!d_n) return n_cap;
    int64_t n = (int64_t)*d_n;
    return n < n_cap ? n : n_cap;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const u32 *__restrict__ in, int64_t n_cap,
                                                              const u32 *d_n, u32 *__restrict__ sums)
{
    int64_t n = eff_n(n_cap, d_n);
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    u32 s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + k * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    u32 tot;
    block_incl_scan<SCAN_THREADS>(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// one block of 1024 threads: exclusive scan of the block sums in place
__global__ void __launch_bounds__(1024) k_scan_sums(u32 *sums, int nb, u32 *d_total)
{
    u32 carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        u32 v = i < nb ? sums[i] : 0u;
        u32 tot;
        u32 inc = block_incl_scan<1024>(v, &tot);
        if (i < nb) sums[i] = carry + inc - v;
        carry += tot;
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const u32 *__restrict__ in, u32 *__restrict__ out,
                                                            int64_t n_cap, const u32 *d_n,
                                                            const u32 *__restrict__ sums)
{
    int64_t n = eff_n(n_cap, d_n);
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    u32 v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    u32 tot;
    u32 run = block_incl_scan<SCAN_THREADS>(s, &tot) - s + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// ------------------------------------------------------------- radix sort
constexpr int RX_BITS = 8;
constexpr int RX = 1 << RX_BITS;
constexpr int RX_WARPS = 8;
constexpr int RX_THREADS = RX_WARPS * 32;
constexpr int RX_ROUNDS = 8;                         // keys per lane
constexpr int RX_TILE = RX_THREADS * RX_ROUNDS;      // 2048 keys per block
constexpr int RX_WARP_SPAN = 32 * RX_ROUNDS;         // 256 consecutive keys per warp

// Per-block digit histogram: hist[digit * nblocks + block]
__global__ void __launch_bounds__(RX_THREADS) k_radix_hist(const u32 *__restrict__ keys, int64_t n_cap,
                                                           const u32 *d_n, int shift, int nblocks,
                                                           u32 *__restrict__ hist)
{
    __shared__ u32 cnt[RX];
    int64_t n = eff_n(n_cap, d_n);
    for (int d = threadIdx.x; d < RX; d += RX_THREADS) cnt[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RX_TILE;
    if (base < n) {
#pragma unroll
        for (int r = 0; r < RX_ROUNDS; ++r) {
            int64_t i = base + r * RX_THREADS + threadIdx.x;
            if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (RX - 1)], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RX; d += RX_THREADS) hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

// Stable scatter.  Warp w owns keys [base + w*256, base + (w+1)*256) and walks
// them in order, 32 at a time; equal digits inside a round are ranked with
// __match_any_sync, so the order of equal keys is preserved.
__global__ void __launch_bounds__(RX_THREADS) k_radix_scatter(const u32 *__restrict__ kin,
                                                              const u32 *__restrict__ vin,
                                                              u32 *__restrict__ kout, u32 *__restrict__ vout,
                                                              int64_t n_cap, const u32 *d_n, int shift,
                                                              int nblocks, const u32 *__restrict__ hist)
{
    __shared__ u32 wcnt[RX_WARPS][RX];
    int64_t n = eff_n(n_cap, d_n);
    int64_t base = (int64_t)blockIdx.x * RX_TILE;
    if (base >= n) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RX_WARPS * RX; d += RX_THREADS) (&wcnt[0][0])[d] = 0;
    __syncthreads();
    u32 k[RX_ROUNDS], v[RX_ROUNDS];
    int dg[RX_ROUNDS];
    const int64_t wbase = base + (int64_t)w * RX_WARP_SPAN;
#pragma unroll
    for (int r = 0; r < RX_ROUNDS; ++r) {
        int64_t i = wbase + r * 32 + lane;
        bool ok = i < n;
        k[r] = ok ? kin[i] : 0u;
        v[r] = ok ? vin[i] : 0u;
        dg[r] = ok ? (int)((k[r] >> shift) & (RX - 1)) : RX;  // RX = no key
        u32 peers = __match_any_sync(0xffffffffu, dg[r]);
        int leader = __ffs(peers) - 1;
        if (ok && lane == leader) wcnt[w][dg[r]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: block offset from the global scan, then exclusive over warps
    for (int d = threadIdx.x; d < RX; d += RX_THREADS) {
        u32 run = hist[(int64_t)d * nblocks + blockIdx.x];
#pragma unroll
        for (int ww = 0; ww < RX_WARPS; ++ww) {
            u32 c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const u32 lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RX_ROUNDS; ++r) {
        u32 peers = __match_any_sync(0xffffffffu, dg[r]);
        int leader = __ffs(peers) - 1;
        u32 pos = 0;
        if (dg[r] < RX) pos = wcnt[w][dg[r]] + __popc(peers & lt);
        __syncwarp();
        if (dg[r] < RX && lane == leader) wcnt[w][dg[r]] += __popc(peers);
        __syncwarp();
        if (dg[r] < RX) {
            kout[pos] = k[r];
            vout[pos] = v[r];
        }
    }
}

} // namespace

gsr_status scan_exclusive(gsr_ctx *ctx, const u32 *in, u32 *out, int64_t n_cap, const u32 *d_n,
                          u32 *d_total, cudaStream_t s)
{
    int64_t nb = ceil_div(n_cap > 0 ? n_cap : 1, SCAN_TILE);
    GSR_TRY(ensure_buf(ctx, ctx->scan_tmp, sizeof(u32) * (size_t)nb));
    u32 *sums = (u32 *)ctx->scan_tmp.p;
    k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n_cap, d_n, sums);
    k_scan_sums<<<1, 1024, 0, s>>>(sums, (int)nb, d_total);
    k_scan_down<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n_cap, d_n, sums);
    ctx->launches += 3;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status radix_sort_pairs(gsr_ctx *ctx, u32 *keys[2], u32 *vals[2], int64_t n_cap, const u32 *d_n,
                            int bits, cudaStream_t s)
{
    int passes = (bits + RX_BITS - 1) / RX_BITS;
    if (passes % 2) ++passes;  // an even count leaves the result in keys[0]
    int64_t nb = ceil_div(n_cap > 0 ? n_cap : 1, RX_TILE);
    size_t hist_words = (size_t)nb * RX;
    GSR_TRY(ensure_buf(ctx, ctx->radix_hist, sizeof(u32) * hist_words));
    u32 *hist = (u32 *)ctx->radix_hist.p;
    int src = 0;
    for (int p = 0; p < passes; ++p) {
        int shift = p * RX_BITS;
        if (shift >= 32) shift = 24;  // padding pass: keys already ordered, stable no-op on top digit
        k_radix_hist<<<(unsigned)nb, RX_THREADS, 0, s>>>(keys[src], n_cap, d_n, shift, (int)nb, hist);
        ctx->launches += 1;
        GSR_LAUNCHED(ctx);
        GSR_TRY(scan_exclusive(ctx, hist, hist, (int64_t)hist_words, nullptr, nullptr, s));
        k_radix_scatter<<<(unsigned)nb, RX_THREADS, 0, s>>>(keys[src], vals[src], keys[src ^ 1], vals[src ^ 1],
                                                           n_cap, d_n, shift, (int)nb, hist);
        ctx->launches += 1;
        GSR_LAUNCHED(ctx);
        src ^= 1;
    }
    return GSR_OK;
}

gsr_status grow_instance_capacity(gsr_ctx *ctx, ViewScratch &V, int64_t c)
{
    if (c <= V.cap_i) return GSR_OK;
    for (int k = 0; k < 2; ++k) {
        GSR_TRY(ensure_buf(ctx, V.tkeys[k], sizeof(u32) * c));
        GSR_TRY(ensure_buf(ctx, V.tvals[k], sizeof(u32) * c));
    }
    // everything the instance sort touches is sized here, so that a captured
    // graph never needs to grow a buffer
    const int64_t hist_words = ceil_div(c, RX_TILE) * RX;
    GSR_TRY(ensure_buf(ctx, ctx->radix_hist, sizeof(u32) * hist_words));
    GSR_TRY(ensure_buf(ctx, ctx->scan_tmp, sizeof(u32) * ceil_div(hist_words, SCAN_TILE)));
    V.cap_i = c;
    return GSR_OK;
}

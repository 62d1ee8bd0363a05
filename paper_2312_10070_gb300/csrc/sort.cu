// sort.cu -- device-wide exclusive scan and stable LSD radix sort of
// (u32 key, u32 value) pairs.  Both read their element count from device
// memory so that a whole frame can be enqueued (and graph-captured) without
// a host round trip; grids are sized by capacity and idle blocks exit.
#include <algorithm>

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
constexpr int RX_MAX_PASSES = 4;
constexpr u32 LB_AGG = 1u << 30, LB_INC = 2u << 30, LB_MASK = (1u << 30) - 1u;
constexpr int LB_SPIN_LIMIT = 1 << 24;               // bounded look-back wait
static_assert(RX_THREADS == RX, "one thread per digit in the look-back and the digit scan");
constexpr int LB_WINDOW = 4;                         // predecessors read per look-back step

// Bounded wait for a look-back word: polls *p (through L2) until one of the
// `ready` bits is set, at most `limit` polls, sleeping briefly between polls
// after the first few so that the blocks still ranking get the issue slots.
// Returns the word, or 0 once the limit is reached, after latching
// GSR_FLAG_TIMEOUT in *status (the caller goes on without the value rather
// than waiting forever).
__device__ __forceinline__ u32 wait_published(const u32 *p, u32 ready, int limit, u32 *status)
{
    for (int spins = 0;; ++spins) {
        const u32 x = __ldcg(p);
        if (x & ready) return x;
        if (spins >= limit) {
            atomicOr(status, GSR_FLAG_TIMEOUT);
            return 0u;
        }
        if (spins >= 4) __nanosleep(32);
    }
}

// Digit totals of every pass at once: ghist[pass * RX + digit] (atomics).
__global__ void __launch_bounds__(RX_THREADS) k_radix_global_hist(const u32 *__restrict__ keys, int64_t n_cap,
                                                                  const u32 *d_n, int passes, u32 *__restrict__ ghist)
{
    __shared__ u32 cnt[RX_MAX_PASSES][RX];
    const int64_t n = eff_n(n_cap, d_n);
    for (int d = threadIdx.x; d < RX_MAX_PASSES * RX; d += RX_THREADS) (&cnt[0][0])[d] = 0;
    __syncthreads();
    // four keys per thread and iteration (16-byte loads; the key arrays are
    // allocation bases, so 16-byte aligned), the last n % 4 keys one by one
    const int64_t n4 = n / 4;
    const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);
    for (int64_t i = (int64_t)blockIdx.x * RX_THREADS + threadIdx.x; i < n4; i += (int64_t)gridDim.x * RX_THREADS) {
        const uint4 k = k4[i];
        for (int p = 0; p < passes; ++p) {
            const int sh = p * RX_BITS;
            atomicAdd(&cnt[p][(k.x >> sh) & (RX - 1)], 1u);
            atomicAdd(&cnt[p][(k.y >> sh) & (RX - 1)], 1u);
            atomicAdd(&cnt[p][(k.z >> sh) & (RX - 1)], 1u);
            atomicAdd(&cnt[p][(k.w >> sh) & (RX - 1)], 1u);
        }
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * RX_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * RX_THREADS) {
        const u32 k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&cnt[p][(k >> (p * RX_BITS)) & (RX - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < passes * RX; d += RX_THREADS) {
        const u32 c = (&cnt[0][0])[d];
        if (c) atomicAdd(&ghist[d], c);
    }
}

// exclusive scan of each pass's 256 digit totals (one block of RX threads per pass)
__global__ void __launch_bounds__(RX) k_radix_digit_base(u32 *ghist)
{
    __shared__ u32 sc[RX];
    u32 *h = ghist + blockIdx.x * RX;
    const u32 v = h[threadIdx.x];
    sc[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < RX; o <<= 1) {
        const u32 t = threadIdx.x >= (unsigned)o ? sc[threadIdx.x - o] : 0u;
        __syncthreads();
        sc[threadIdx.x] += t;
        __syncthreads();
    }
    h[threadIdx.x] = sc[threadIdx.x] - v;
}

// Lanes of the warp whose digit equals this lane's: one ballot per digit bit
// (BITS = RX_BITS + 1 when digit RX marks "no key" in a partial tile).
template <int BITS>
__device__ __forceinline__ u32 digit_peers(u32 dg)
{
    u32 peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (dg >> b) & 1u;
        const u32 m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

// One stable pass.  Blocks take 2048-key tiles in launch order (atomic ticket,
// so every tile a block waits for belongs to a block that already runs);
// each warp ranks its consecutive keys in order with digit_peers (keeping
// each key's rank among the warp's keys of its digit); the
// block publishes its digit counts, looks back over the preceding tiles for
// their running totals, stages its keys in shared memory in digit order and
// writes them out so that equal digits land in consecutive addresses.
template <int ROUNDS>
__global__ void __launch_bounds__(RX_THREADS, 4) k_radix_onesweep(const u32 *__restrict__ kin, const u32 *__restrict__ vin,
                                                               u32 *__restrict__ kout, u32 *__restrict__ vout,
                                                               int64_t n_cap, const u32 *d_n, int shift,
                                                               const u32 *__restrict__ digit_base,
                                                               u32 *__restrict__ lookback, u32 *ticket,
                                                               u32 *status)
{
    __shared__ u32 wcnt[RX_WARPS][RX];
    constexpr int TILE = RX_THREADS * ROUNDS, SPAN = 32 * ROUNDS;
    __shared__ u32 s_key[TILE], s_val[TILE];
    __shared__ u32 s_gpos[RX];
    __shared__ int s_tile;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(ticket, 1u);
    for (int d = threadIdx.x; d < RX_WARPS * RX; d += RX_THREADS) (&wcnt[0][0])[d] = 0;
    __syncthreads();
    const int tile = s_tile;
    const int64_t n = eff_n(n_cap, d_n);
    const int64_t base = (int64_t)tile * TILE;
    if (base >= n) return;  // no key in this tile (and none in any later tile)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    u32 k[ROUNDS], v[ROUNDS], rk[ROUNDS];
    const int64_t wbase = base + (int64_t)w * SPAN;
    const u32 lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        k[r] = i < n ? kin[i] : 0u;
        v[r] = i < n ? vin[i] : 0u;
    }
    const bool full = base + TILE <= n;  // every lane holds a key in every round
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const bool ok = wbase + r * 32 + lane < n;
        const u32 dg = ok ? (k[r] >> shift) & (RX - 1) : (u32)RX;  // RX = no key
        const u32 peers = full ? digit_peers<RX_BITS>(dg) : digit_peers<RX_BITS + 1>(dg);
        // rank of this key among the warp's keys of its digit, in input order
        const u32 before = ok ? wcnt[w][dg] : 0u;
        rk[r] = ok ? before + __popc(peers & lt) : ~0u;  // ~0: no key
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wcnt[w][dg] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit (thread d): block total, publish, look back
    const int d = threadIdx.x;
    u32 tot = 0;
#pragma unroll
    for (int ww = 0; ww < RX_WARPS; ++ww) tot += wcnt[ww][d];
    u32 *my = lookback + (int64_t)tile * RX + d;
    if (tile == 0) {
        __stcg(my, LB_INC | tot);
    } else {
        __stcg(my, LB_AGG | tot);
    }
    u32 prefix = 0;
    if (tile > 0) {
        // LB_WINDOW predecessors are read at once (one L2 round trip per
        // window); a word not yet published when read is then waited for.  A
        // word read as an aggregate may have become inclusive since, and
        // using the aggregate only extends the walk.  Tile 0 publishes an
        // inclusive value, so the walk ends at j = 0 at the latest.
        int j = tile - 1;
        bool done = false;
        while (!done) {
            u32 x[LB_WINDOW];
#pragma unroll
            for (int k = 0; k < LB_WINDOW; ++k) x[k] = j - k >= 0 ? __ldcg(lookback + (int64_t)(j - k) * RX + d) : 0u;
#pragma unroll
            for (int k = 0; k < LB_WINDOW; ++k) {
                if (done) break;
                u32 v = x[k];
                if (!(v & ~LB_MASK)) {
                    v = wait_published(lookback + (int64_t)(j - k) * RX + d, ~LB_MASK, LB_SPIN_LIMIT, status);
                    if (v == 0u) {  // a predecessor never published: flagged, give up
                        done = true;
                        break;
                    }
                }
                prefix += v & LB_MASK;
                if ((v & ~LB_MASK) == LB_INC) done = true;
            }
            j -= LB_WINDOW;
        }
        __stcg(my, LB_INC | (prefix + tot));
    }
    // block-local digit starts (exclusive scan over digits of tot): a
    // shuffle scan within each warp of 32 digits, then the warp totals
    {
        __shared__ u32 s_wt[RX / 32];
        u32 x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wt[w] = x;
        __syncthreads();
        for (int k = 0; k < w; ++k) x += s_wt[k];
        const u32 lstart = x - tot;
        s_gpos[d] = digit_base[d] + prefix - lstart;  // global slot of local position i: s_gpos + i
        u32 run = lstart;  // per-warp starts inside the block
#pragma unroll
        for (int ww = 0; ww < RX_WARPS; ++ww) {
            const u32 c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        if (rk[r] != ~0u) {
            const u32 pos = wcnt[w][(k[r] >> shift) & (RX - 1)] + rk[r];  // the warp's start for the digit + rank
            s_key[pos] = k[r];
            s_val[pos] = v[r];
        }
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)TILE, n - base);
    for (int i = threadIdx.x; i < cnt; i += RX_THREADS) {
        const u32 key = s_key[i];
        const int dd = (int)((key >> shift) & (RX - 1));
        const u32 gp = s_gpos[dd] + (u32)i;
        kout[gp] = key;
        vout[gp] = s_val[i];
    }
}

// Failure-detection check: one warp runs the look-back's bounded wait on a
// word that nothing publishes, so the wait expires and latches the timeout.
__global__ void k_wait_unpublished(const u32 *word, int limit, u32 *status)
{
    wait_published(word, ~LB_MASK, limit, status);
}

} // namespace

gsr_status lookback_wait_check(gsr_ctx *ctx, const u32 *word, int32_t polls, u32 *status, cudaStream_t s)
{
    k_wait_unpublished<<<1, 32, 0, s>>>(word, polls, status);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status scan_exclusive(gsr_ctx *ctx, const u32 *in, u32 *out, int64_t n_cap, const u32 *d_n,
                          u32 *d_total, cudaStream_t s, DevBuf *tmp)
{
    int64_t nb = ceil_div(n_cap > 0 ? n_cap : 1, SCAN_TILE);
    DevBuf &sb = tmp ? *tmp : ctx->scan_tmp;
    GSR_TRY(ensure_buf(ctx, sb, sizeof(u32) * (size_t)nb));
    u32 *sums = (u32 *)sb.p;
    k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n_cap, d_n, sums);
    k_scan_sums<<<1, 1024, 0, s>>>(sums, (int)nb, d_total);
    k_scan_down<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n_cap, d_n, sums);
    ctx->launches += 3;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status radix_sort_pairs(gsr_ctx *ctx, u32 *keys[2], u32 *vals[2], int64_t n_cap, const u32 *d_n,
                            int bits, cudaStream_t s, DevBuf *hist)
{
    DevBuf &hb_buf = hist ? *hist : ctx->radix_hist;
    int passes = (bits + RX_BITS - 1) / RX_BITS;
    if (passes % 2) ++passes;  // an even count leaves the result in keys[0]
    if (passes > RX_MAX_PASSES) passes = RX_MAX_PASSES;
    // 2048-key tiles for every size (with the windowed look-back, 1024-key
    // tiles for the small depth sorts measured 3 us slower per frame)
    const int64_t nb = ceil_div(n_cap > 0 ? n_cap : 1, RX_TILE);
    // layout of radix_hist: [ghist: passes * RX][per pass: lookback nb * RX + ticket]
    const int64_t lb_words = nb * RX + 32;
    const size_t words = (size_t)RX_MAX_PASSES * RX + (size_t)passes * lb_words;
    GSR_TRY(ensure_buf(ctx, hb_buf, sizeof(u32) * words));
    u32 *ghist = (u32 *)hb_buf.p;
    u32 *lb0 = ghist + RX_MAX_PASSES * RX;
    GSR_CUDA(ctx, cudaMemsetAsync(ghist, 0, sizeof(u32) * words, s));
    const unsigned hb = (unsigned)std::min<int64_t>(nb, 2 * 152);
    k_radix_global_hist<<<hb, RX_THREADS, 0, s>>>(keys[0], n_cap, d_n, passes, ghist);
    k_radix_digit_base<<<passes, RX, 0, s>>>(ghist);
    ctx->launches += 2;
    GSR_LAUNCHED(ctx);
    GSR_TRY(ensure_buf(ctx, ctx->view.counters, sizeof(u32) * CNT_WORDS));
    u32 *status = (u32 *)ctx->view.counters.p + CNT_STATUS;
    int src = 0;
    for (int p = 0; p < passes; ++p) {
        u32 *lb = lb0 + (size_t)p * lb_words;
        k_radix_onesweep<RX_ROUNDS><<<(unsigned)nb, RX_THREADS, 0, s>>>(keys[src], vals[src], keys[src ^ 1], vals[src ^ 1],
                                                                        n_cap, d_n, p * RX_BITS, ghist + p * RX, lb,
                                                                        lb + nb * RX, status);
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
    const int64_t words = RX_MAX_PASSES * RX + RX_MAX_PASSES * (ceil_div(c, RX_TILE) * RX + 32);
    GSR_TRY(ensure_buf(ctx, V.radix_hist, sizeof(u32) * words));
    V.cap_i = c;
    return GSR_OK;
}

// fd_batch.cu -- many 2D shots in one persistent, dependency-driven launch.
//
// The time step is the one of fd_kernels.cu (the paper's section 7 routine
// sequence, fused); what changes is the schedule.  Instead of one launch per
// shot and time step, one cooperative launch of resident CTAs walks a table of
// work items (shot, tile).  Each item keeps a completed-step counter in global
// memory: a tile may compute step k+1 once it and its four neighbours have
// completed step k.  That single rule orders both hazards of the two rotating
// buffers: the halo it reads (written by the neighbours at step k) and the
// region it overwrites (read as halo by the neighbours at step k).
//
// Inside a CTA one producer lane waits on the counters (bounded spins), then
// issues the TMA loads of the haloed P tile and the Pold and w tiles into a
// ring of stages; the consumer warps compute the tile with the shared arithmetic
// of stencil.cuh, write Pn, the tile's receivers and the source, and publish
// the counter with release semantics.  Items are visited group by group; all
// time steps of a launch are done on one group before the next, so a group
// whose fields fit in L2 stays resident while it steps.
//
// The launch carries no per-launch arguments: the step base is a counter in
// device memory advanced by the last CTA to finish, so one captured graph node
// is replayed until every shot has reached its target.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fd.h"
#include "fd_internal.h"
#include "fd_model.h"
#include "fd_trace.h"
#include "ptx.cuh"
#include "stencil.cuh"

namespace fdk {

struct ShotDesc {
    CUtensorMap halo[2];   // haloed P box over buf[i]
    CUtensorMap tile[2];   // tile box over buf[i] (as Pold)
    CUtensorMap wmap;
    float *buf[2];
    const float *ax, *az;
    const float *amp;      // dt^2 S(t_n) / h^2 per absolute step
    float *traces;
    int namp, trace_rows, nrec;
    int nx, nz, px;
    int n0, cur0, target, has_sponge;
    int src_on, sx, sz;
};

struct BatchItem {
    int shot, x0, z0;
    int nb[4];             // neighbour items (left, right, up, down), -1 at the grid edge
    int rec_begin, rec_end;
};

struct BatchRec {
    int local;             // (z - z0) * TX + (x - x0) within the tile
    int r;                 // receiver index of the shot
};

struct BatchState {
    int launch;            // launches completed in the current run
    unsigned done;         // CTAs finished in the current launch
};

struct BatchParams {
    const ShotDesc *shots;
    const BatchItem *items;
    const BatchRec *recs;
    int *counters;         // per item: steps completed in the current run
    const int *group_begin;
    int ngroups;
    int K;                 // steps per launch
    BatchState *state;
    float c1, c2, c3, c4;
    int *err;
    int stall_item;        // test hook: this item never runs (-1: none)
};

// What the consumers need about the item in a ring stage; written by the
// producer before it arms the stage's barrier, so consumers read only shared
// memory.  item < 0 marks the end of the work.
struct StageMeta {
    float *out;            // Pn destination (the shot's Pold buffer)
    float *trace_row;      // traces + n * nrec, or null when no row is recorded
    int item, x0, z0, nx, nz, px;
    int rec_begin, rec_end;
    int src_local;         // the source's (z - z0) * TX + (x - x0), or -1
    float src_amp;
    int has_sponge;
    int cs;                // the step this stage computes (run-relative)
};

// A stage's receiver row, handed from before the stage barrier to after it.
struct GatherRow {
    float *row;            // trace row, or null
    int begin, end;        // receiver range of the item
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Order this thread's earlier generic-proxy accesses (the acquire of a
// neighbour's counter) before its later async-proxy (TMA) reads of global memory.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// AND of v over the nthreads threads of named barrier id (all of them must call it).
__device__ __forceinline__ bool named_and(int id, int nthreads, bool v)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((int)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until item i and its neighbours have completed v steps: the five
// counters are read together (independent relaxed loads), and one acquire
// fence orders the later reads after them.  False if the cycle budget runs
// out or *abort is raised.
__device__ __forceinline__ bool wait_deps(const int *counters, int i, const int (&nb)[4], int v,
                                          volatile int *abort, const volatile int *err)
{
    long long t0 = -1;
    for (;;) {
        const int c0 = ld_relaxed(&counters[i]);
        const int c1 = nb[0] >= 0 ? ld_relaxed(&counters[nb[0]]) : v;
        const int c2 = nb[1] >= 0 ? ld_relaxed(&counters[nb[1]]) : v;
        const int c3 = nb[2] >= 0 ? ld_relaxed(&counters[nb[2]]) : v;
        const int c4 = nb[3] >= 0 ? ld_relaxed(&counters[nb[3]]) : v;
        if (min(min(c0, c1), min(min(c2, c3), c4)) >= v)
            break;
        if (t0 < 0)
            t0 = clock64();
        else if (*abort || *err || clock64() - t0 > kWaitLimitCycles)
            return false;    // own budget spent, or another CTA already gave up
        __nanosleep(32);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return true;
}

template <int TX, int TZ, int S>
__global__ void __launch_bounds__(TX / 4 * TZ + 32) batch2d_kernel(const BatchParams bp)
{
    constexpr int QX = TX / 4;
    constexpr int NC = QX * TZ;
    constexpr int NCW = NC / 32;
    constexpr int HX = TX + 8;
    constexpr int HZ = TZ + 8;
    constexpr int PBOX = HX * HZ;
    constexpr int TBOX = TX * TZ;
    constexpr uint32_t BYTES = (PBOX + 2 * TBOX) * 4;
    static_assert(NC % 32 == 0, "consumers must fill warps");
    static_assert((PBOX * 4) % 128 == 0 && (TBOX * 4) % 128 == 0, "boxes keep 128-byte alignment");

    extern __shared__ __align__(128) unsigned char smem[];
    float *sP = reinterpret_cast<float *>(smem);
    float *sO = sP + S * PBOX;
    float *sW = sO + S * TBOX;
    float *sAx = sW + S * TBOX;             // [S][TX] sponge slice along x
    float *sAz = sAx + S * TX;              // [S][TZ] sponge slice along z
    float *sPn = sAz + S * TZ;              // [2][TBOX] results, for the receivers
    uint64_t *full = reinterpret_cast<uint64_t *>(sPn + 2 * TBOX);
    uint64_t *empty = full + S;
    StageMeta *meta = reinterpret_cast<StageMeta *>(empty + S);
    __shared__ int s_abort;
    __shared__ GatherRow s_gather[2];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int launch = *reinterpret_cast<volatile int *>(&bp.state->launch);

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    if (warp == NCW) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int k = 0;
            bool good = true;
            for (int g = 0; good && g < bp.ngroups; ++g) {
                const int ib = bp.group_begin[g], ie = bp.group_begin[g + 1];
                for (int sw = 0; good && sw < bp.K; ++sw) {
                    const int cs = launch * bp.K + sw;
                    BatchItem nxt;
                    if (ib + (int)blockIdx.x < ie)
                        nxt = bp.items[ib + blockIdx.x];
                    for (int i = ib + blockIdx.x; i < ie; i += gridDim.x) {
                        const BatchItem it = nxt;
                        if (i + (int)gridDim.x < ie)
                            nxt = bp.items[i + gridDim.x];   // prefetch the next descriptor
                        const ShotDesc &sd = bp.shots[it.shot];
                        if (cs >= sd.target || i == bp.stall_item)
                            continue;
                        good = wait_deps(bp.counters, i, it.nb, cs, &s_abort, bp.err);
                        const int slot = k % S;
                        if (good && k >= S)
                            good = mbar_wait(&empty[slot], ((k / S) - 1) & 1, &s_abort);
                        if (!good)
                            break;
                        fence_proxy_async_global();
                        const int pb = (sd.cur0 + cs) & 1;
                        const int n = sd.n0 + cs;
                        StageMeta &mt = meta[slot];
                        mt.out = sd.buf[pb ^ 1];
                        mt.trace_row = (it.rec_begin < it.rec_end && n < sd.trace_rows)
                                           ? sd.traces + (size_t)n * sd.nrec
                                           : nullptr;
                        mt.item = i;
                        mt.cs = cs;
                        mt.x0 = it.x0;
                        mt.z0 = it.z0;
                        mt.nx = sd.nx;
                        mt.nz = sd.nz;
                        mt.px = sd.px;
                        mt.rec_begin = it.rec_begin;
                        mt.rec_end = it.rec_end;
                        const bool src_here = sd.src_on && n < sd.namp && sd.sx >= it.x0 && sd.sx < it.x0 + TX &&
                                              sd.sz >= it.z0 && sd.sz < it.z0 + TZ;
                        mt.src_local = src_here ? (sd.sz - it.z0) * TX + (sd.sx - it.x0) : -1;
                        mt.src_amp = src_here ? sd.amp[n] : 0.f;
                        mt.has_sponge = sd.has_sponge;
                        mbar_arrive_expect_tx(&full[slot], BYTES + (sd.has_sponge ? (TX + TZ) * 4 : 0));
                        tma_load_2d(sP + slot * PBOX, &sd.halo[pb], &full[slot], it.x0 - 4, it.z0 - 4);
                        tma_load_2d(sO + slot * TBOX, &sd.tile[pb ^ 1], &full[slot], it.x0, it.z0);
                        tma_load_2d(sW + slot * TBOX, &sd.wmap, &full[slot], it.x0, it.z0);
                        if (sd.has_sponge) {
                            bulk_load(sAx + slot * TX, sd.ax + it.x0, TX * 4, &full[slot]);
                            bulk_load(sAz + slot * TZ, sd.az + it.z0, TZ * 4, &full[slot]);
                        }
                        ++k;
                    }
                }
            }
            const int slot = k % S;
            if (good && (k < S || mbar_wait(&empty[slot], ((k / S) - 1) & 1, &s_abort))) {
                // end marker for the consumers (every issued stage is waited on by
                // them before the CTA can exit, so no copy outlives the CTA)
                meta[slot].item = -1;
                mbar_arrive(&full[slot]);
            } else {
                // abort: consumers leave on the flag; stay until the copies into
                // this CTA's shared memory have landed (bounded)
                raise_error(bp.err, &s_abort, kDevErrTimeout);
                int never = 0;
                for (int q = max(0, k - S); q < k; ++q)
                    mbar_wait(&full[q % S], (q / S) & 1, &never, kWaitLimitCycles / 8);
            }
        }
    } else {
        // ------------------------------------------------------------ consumers
        // One named barrier per stage, which also votes: every consumer thread
        // reaches it, including a warp whose wait gave up (it skips the work), so
        // all take the same decision to go on or stop and none is left waiting.
        const int tx = tid % QX;
        const int tz = tid / QX;
        for (int k = 0;; ++k) {
            const int slot = k % S;
            float *pn = sPn + (k & 1) * TBOX;
            const bool good = __all_sync(0xffffffffu, mbar_wait(&full[slot], (k / S) & 1, &s_abort));
            bool work = false;
            if (good) {
                const StageMeta &mt = meta[slot];
                work = mt.item >= 0;
                if (work) {
                    const int x = mt.x0 + 4 * tx;
                    const int z = mt.z0 + tz;
                    float axv[4] = {0.f, 0.f, 0.f, 0.f};
                    float azv = 0.f;
                    if (mt.has_sponge) {
                        const float4 a4 = *reinterpret_cast<const float4 *>(sAx + slot * TX + 4 * tx);
                        axv[0] = a4.x;
                        axv[1] = a4.y;
                        axv[2] = a4.z;
                        axv[3] = a4.w;
                        azv = sAz[slot * TZ + tz];
                    }
                    float2 r[2], lp[2];
                    tile2d_update<TX>(sP + slot * PBOX, sO + slot * TBOX, sW + slot * TBOX, tx, tz, axv, azv, bp.c1,
                                      bp.c2, bp.c3, bp.c4, r, lp);
                    const int local = tz * TX + 4 * tx;
                    if ((unsigned)(mt.src_local - local) < 4u)
                        add_source4(r, mt.src_local - local, mt.src_amp);
                    if (z < mt.nz && x < mt.nx)
                        store4(mt.out + (size_t)z * mt.px + x, r, mt.nx - x);
                    if (mt.rec_begin < mt.rec_end)
                        *reinterpret_cast<float4 *>(pn + local) = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
                    if (tid == 0)
                        s_gather[k & 1] = GatherRow{mt.trace_row, mt.rec_begin, mt.rec_end};
                }
            } else {
                raise_error(bp.err, &s_abort, kDevErrTimeout);
            }
            if (!named_and(1, NC, work))
                break;   // end marker, or some consumer gave up
            if (tid == 0) {
                // the slot is still this stage's until the empty arrive below
                const int item = meta[slot].item, cs = meta[slot].cs;
                __threadfence();
                st_release(&bp.counters[item], cs + 1);
                mbar_arrive(&empty[slot]);
            }
            // Receivers of this stage, from the double-buffered result tile and
            // row record: stage k+1 writes the other ones, and stage k+2 passes
            // stage k+1's barrier only when every thread has finished reading.
            const GatherRow gr = s_gather[k & 1];
            if (gr.row)
                for (int q = gr.begin + tid; q < gr.end; q += NC)
                    gr.row[bp.recs[q].r] = pn[bp.recs[q].local];
        }
    }

    // the last CTA to finish advances the launch counter for the next replay
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&bp.state->done, 1u) == gridDim.x - 1) {
            bp.state->done = 0;
            bp.state->launch = launch + 1;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------- wide schedule
//
// One ordinary launch per time step over the tiles of up to kWideMax shots, a
// CTA per (shot, tile).  Everything a CTA needs -- its shot's three tensor maps,
// pointers, extents, source and receivers -- travels in the launch's parameter
// block, so a CTA finds its shot by a binary search over the shots' first tiles
// in parameter space and issues its TMA loads at once, with no dependent global
// loads before them.  The per-tile arithmetic is the single-shot 2D step's
// (stencil.cuh), so shots are bitwise the same as alone.  No CTA waits on
// another: the launch boundary orders the steps.

constexpr int kWideMax = 64;

struct WideShot {
    float *out;               // Pn destination (the shot's Pold buffer)
    const float *P;           // level n (read by the receiver gather)
    const float *ax, *az;
    float *trace_prev;        // the row owed for level n, or null
    const int64_t *rec_idx;
    int nrec;
    int nx, nz, px;
    int tiles_x;
    int tile_begin;           // first CTA of this shot
    int has_sponge, src_on, sx, sz;
    float src_amp;
};

struct WideParams {
    CUtensorMap halo[kWideMax];   // haloed P box over level n
    CUtensorMap tile[kWideMax];   // Pold tile box
    CUtensorMap wmap[kWideMax];
    WideShot shot[kWideMax];
    int nshots;
    float c1, c2, c3, c4;
    int *err;
};

// A CTA owns a column of up to ZT tiles stacked along z in one shot and walks
// down it through a two-stage TMA ring: the load of tile i + 1 is in flight
// while tile i is computed.  ZT = 1 is one tile per CTA.
template <int TX, int TZ, int ZT>
__global__ void __launch_bounds__(TX / 4 * TZ) wide2d_kernel(const __grid_constant__ WideParams prm)
{
    constexpr int QX = TX / 4;
    constexpr int HX = TX + 8;
    constexpr int HZ = TZ + 8;
    constexpr int NS = ZT > 1 ? 2 : 1;
    constexpr uint32_t BYTES = (HX * HZ + 2 * TX * TZ) * 4;
    __shared__ __align__(128) float sP[NS][HX * HZ];
    __shared__ __align__(128) float sO[NS][TX * TZ];
    __shared__ __align__(128) float sW[NS][TX * TZ];
    __shared__ __align__(8) uint64_t bar[NS];
    __shared__ int s_abort;

    // the shot of this CTA: the last s with shot[s].tile_begin <= blockIdx.x
    int lo = 0, hi = prm.nshots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prm.shot[mid].tile_begin <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int s = lo;
    const WideShot &sh = prm.shot[s];
    const int c = blockIdx.x - sh.tile_begin;          // CTA within the shot
    const int tiles_z = (sh.nz + TZ - 1) / TZ;
    const int x0 = (c % sh.tiles_x) * TX;
    const int tz0 = (c / sh.tiles_x) * ZT;              // first tile row of this column
    const int nt = min(ZT, tiles_z - tz0);
    const int tid = threadIdx.x;

    auto issue = [&](int i) {
        const int st = i % NS;
        const int z0 = (tz0 + i) * TZ;
        mbar_arrive_expect_tx(&bar[st], BYTES);
        tma_load_2d(sP[st], &prm.halo[s], &bar[st], x0 - 4, z0 - 4);
        tma_load_2d(sO[st], &prm.tile[s], &bar[st], x0, z0);
        tma_load_2d(sW[st], &prm.wmap[s], &bar[st], x0, z0);
    };
    if (tid == 0) {
        for (int st = 0; st < NS; ++st)
            mbar_init(&bar[st], 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < min(NS, nt); ++i)
            issue(i);
    // receivers of this shot's previous step, spread over the shot's CTAs
    if (sh.trace_prev) {
        const int ncta = sh.tiles_x * ((tiles_z + ZT - 1) / ZT);
        for (int r = c * blockDim.x + tid; r < sh.nrec; r += ncta * blockDim.x)
            sh.trace_prev[r] = sh.P[sh.rec_idx[r]];
    }

    const int tx = tid % QX;
    const int tz = tid / QX;
    const int x = x0 + 4 * tx;
    float axv[4] = {0.f, 0.f, 0.f, 0.f};
    if (sh.has_sponge) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            axv[e] = x + e < sh.px ? sh.ax[x + e] : 0.f;
    }
    for (int i = 0; i < nt; ++i) {
        const int st = i % NS;
        const int z = (tz0 + i) * TZ + tz;
        const float azv = sh.has_sponge && z < sh.nz ? sh.az[z] : 0.f;
        const bool ok = __syncthreads_and(mbar_wait(&bar[st], (i / NS) & 1, &s_abort));
        if (!ok) {
            if (tid == 0) {
                raise_error(prm.err, &s_abort, kDevErrTimeout);
                // the other stage's copy may still be in flight: wait for it (bounded)
                int never = 0;
                if (NS > 1 && i + 1 < nt)
                    mbar_wait(&bar[(i + 1) % NS], ((i + 1) / NS) & 1, &never, kWaitLimitCycles / 8);
            }
            return;
        }
        float2 r[2], lp[2];
        tile2d_update<TX>(sP[st], sO[st], sW[st], tx, tz, axv, azv, prm.c1, prm.c2, prm.c3, prm.c4, r, lp);
        if (sh.src_on && z == sh.sz && (unsigned)(sh.sx - x) < 4u)
            add_source4(r, sh.sx - x, sh.src_amp);
        if (z < sh.nz && x < sh.nx)
            store4(sh.out + (size_t)z * sh.px + x, r, sh.nx - x);
        if (NS > 1 && i + NS < nt) {
            __syncthreads();   // every thread has read stage st
            if (tid == 0) {
                fence_proxy_async_shared();
                issue(i + NS);
            }
        }
    }
}

// Compiled tile variants: 0 = 64 x 16, 1 = 64 x 32, 2 = 128 x 16.
constexpr int kBatchStages = 3;
struct Variant {
    int tx, tz;
    const void *fn;
    int threads;
    size_t smem;
    bool wide = false;   // one launch per time step (wide2d_kernel) instead of the persistent kernel
    int zt = 1;          // wide: tiles stacked along z per CTA
};

template <int TX, int TZ>
static Variant variant()
{
    constexpr int PBOX = (TX + 8) * (TZ + 8);
    constexpr int TBOX = TX * TZ;
    const size_t smem = (size_t)(kBatchStages * (PBOX + 2 * TBOX + TX + TZ) + 2 * TBOX) * 4 + 2 * kBatchStages * 8 +
                        kBatchStages * sizeof(StageMeta);
    return Variant{TX, TZ, (const void *)batch2d_kernel<TX, TZ, kBatchStages>, TX / 4 * TZ + 32, smem};
}

template <int TX, int TZ, int ZT>
static Variant wide_variant()
{
    Variant v{TX, TZ, (const void *)wide2d_kernel<TX, TZ, ZT>, TX / 4 * TZ, 0, true};
    v.zt = ZT;
    return v;
}

// Tile variants: 0 = 64 x 16, 1 = 64 x 32, 2 = 128 x 16 (persistent kernel);
// 3 = 64 x 16, 4 = 64 x 32, 5 / 6 / 7 = 64 x 16 with 4 / 8 / 16 tiles stacked
// along z per CTA (one launch per time step).
static Variant get_variant(int tile)
{
    switch (tile) {
    case 1:
        return variant<64, 32>();
    case 2:
        return variant<128, 16>();
    case 3:
        return wide_variant<64, 16, 1>();
    case 4:
        return wide_variant<64, 32, 1>();
    case 5:
        return wide_variant<64, 16, 4>();
    case 6:
        return wide_variant<64, 16, 8>();
    case 7:
        return wide_variant<64, 16, 16>();
    default:
        return variant<64, 16>();
    }
}

}  // namespace fdk

using namespace fdk;

// ------------------------------------------------------------------------ host

struct fd_batch {
    std::vector<fd_model *> models;
    int device = 0;
    cudaStream_t stream = nullptr;   // owned by the batch
    fd_batch_tuning tun{0, 2000, 0, 96};
    bool built = false;     // tables match the tuning
    ShotDesc *d_shots = nullptr;
    BatchItem *d_items = nullptr;
    BatchRec *d_recs = nullptr;
    int *d_counters = nullptr;
    int *d_group = nullptr;
    BatchState *d_state = nullptr;
    int *d_err = nullptr;
    int nitems = 0, ngroups = 0, grid = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<ShotDesc> shots;   // host copy (tensor maps, pointers)
    std::vector<int> group_shot;   // first shot of each group, then the shot count
    WideParams wide{};             // parameter block of the wide schedule's launches
    Wide3Params wide3{};           // ... and of the batched 3D schedule's
    int stall_item = -1;           // fd_batch_set_fault
};

static void free_tables(fd_batch *b)
{
    cudaFree(b->d_shots);
    cudaFree(b->d_items);
    cudaFree(b->d_recs);
    cudaFree(b->d_counters);
    cudaFree(b->d_group);
    b->d_shots = nullptr;
    b->d_items = nullptr;
    b->d_recs = nullptr;
    b->d_counters = nullptr;
    b->d_group = nullptr;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->built = false;
}

// Build the item table, receiver lists, groups and per-shot descriptors for
// the current tuning (shot-dependent fields n0 / cur0 / target are set per run).
static fd_status build_tables(fd_batch *b)
{
    free_tables(b);
    const Variant v = get_variant(b->tun.tile);
    std::vector<BatchItem> items;
    std::vector<BatchRec> recs;
    std::vector<int> group{0};
    b->group_shot.assign(1, 0);
    const double budget = b->tun.group_mb > 0 ? b->tun.group_mb * 1048576.0 : 1e300;
    double in_group = 0.0;
    b->shots.assign(b->models.size(), ShotDesc{});
    for (size_t s = 0; s < b->models.size(); ++s) {
        fd_model *m = b->models[s];
        ShotDesc &d = b->shots[s];
        bool ok = true;
        for (int i = 0; i < 2; ++i) {
            ok = ok && make_map(&d.halo[i], m->buf[i], 2, m->nx, 1, m->nz, m->px, v.tx + 8, v.tz + 8);
            ok = ok && make_map(&d.tile[i], m->buf[i], 2, m->nx, 1, m->nz, m->px, v.tx, v.tz);
            d.buf[i] = m->buf[i];
        }
        ok = ok && make_map(&d.wmap, m->w, 2, m->nx, 1, m->nz, m->px, v.tx, v.tz);
        if (!ok)
            return fail(FD_ECUDA, "cuTensorMapEncodeTiled failed for batch shot %zu", s);
        d.ax = m->ax;
        d.az = m->az;
        d.nx = m->nx;
        d.nz = m->nz;
        d.px = m->px;
        d.has_sponge = m->has_sponge;
        // shot grouping by field bytes (P, Pold, w)
        const double bytes = 3.0 * m->pitched * sizeof(float);
        if (s > 0 && in_group + bytes > budget) {
            group.push_back((int)items.size());
            b->group_shot.push_back((int)s);
            in_group = 0.0;
        }
        in_group += bytes;
        // tiles of this shot, row-major; neighbours are items of the same shot
        const int tx_n = (m->nx + v.tx - 1) / v.tx, tz_n = (m->nz + v.tz - 1) / v.tz;
        const int base = (int)items.size();
        std::vector<std::vector<BatchRec>> tile_recs((size_t)tx_n * tz_n);
        for (int r = 0; r < m->nrec; ++r) {
            const int64_t di = m->rec_dense[r];
            const int ix = (int)(di % m->nx), iz = (int)(di / m->nx);
            const int t = (iz / v.tz) * tx_n + ix / v.tx;
            tile_recs[t].push_back(BatchRec{(iz % v.tz) * v.tx + ix % v.tx, r});
        }
        for (int tz = 0; tz < tz_n; ++tz)
            for (int tx = 0; tx < tx_n; ++tx) {
                BatchItem it{};
                it.shot = (int)s;
                it.x0 = tx * v.tx;
                it.z0 = tz * v.tz;
                it.nb[0] = tx > 0 ? base + tz * tx_n + tx - 1 : -1;
                it.nb[1] = tx + 1 < tx_n ? base + tz * tx_n + tx + 1 : -1;
                it.nb[2] = tz > 0 ? base + (tz - 1) * tx_n + tx : -1;
                it.nb[3] = tz + 1 < tz_n ? base + (tz + 1) * tx_n + tx : -1;
                const auto &tr = tile_recs[(size_t)tz * tx_n + tx];
                it.rec_begin = (int)recs.size();
                recs.insert(recs.end(), tr.begin(), tr.end());
                it.rec_end = (int)recs.size();
                items.push_back(it);
            }
    }
    group.push_back((int)items.size());
    b->group_shot.push_back((int)b->models.size());
    b->nitems = (int)items.size();
    b->ngroups = (int)group.size() - 1;
    FD_CUDA(cudaMalloc((void **)&b->d_shots, b->shots.size() * sizeof(ShotDesc)), "batch allocation");
    FD_CUDA(cudaMalloc((void **)&b->d_items, std::max<size_t>(1, items.size()) * sizeof(BatchItem)), "batch allocation");
    FD_CUDA(cudaMalloc((void **)&b->d_recs, std::max<size_t>(1, recs.size()) * sizeof(BatchRec)), "batch allocation");
    FD_CUDA(cudaMalloc((void **)&b->d_counters, std::max(1, b->nitems) * sizeof(int)), "batch allocation");
    FD_CUDA(cudaMalloc((void **)&b->d_group, group.size() * sizeof(int)), "batch allocation");
    FD_CUDA(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice), "batch upload");
    if (!recs.empty())
        FD_CUDA(cudaMemcpy(b->d_recs, recs.data(), recs.size() * sizeof(BatchRec), cudaMemcpyHostToDevice), "batch upload");
    FD_CUDA(cudaMemcpy(b->d_group, group.data(), group.size() * sizeof(int), cudaMemcpyHostToDevice), "batch upload");

    if (v.wide) {
        b->built = true;   // the wide schedule needs only the descriptors and the groups
        return FD_OK;
    }
    // resident grid
    FD_CUDA(cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem), "kernel attributes");
    int per_sm = 0, sms = 0;
    FD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.fn, v.threads, v.smem), "occupancy");
    FD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "device attribute");
    if (per_sm < 1)
        return fail(FD_ECUDA, "batch kernel does not fit on an SM");
    if (b->tun.ctas_per_sm > 0)
        per_sm = std::min(per_sm, b->tun.ctas_per_sm);
    b->grid = sms * per_sm;
    b->built = true;
    return FD_OK;
}

extern "C" fd_status fd_batch_create(fd_model *const *models, int nmodels, fd_batch **out)
{
    if (!out || !models || nmodels < 1)
        return fail(FD_EINVAL, "fd_batch_create: bad arguments");
    *out = nullptr;
    for (int i = 0; i < nmodels; ++i) {
        if (!models[i])
            return fail(FD_EINVAL, "fd_batch_create: model %d is NULL", i);
        if (models[i]->d.ndim != models[0]->d.ndim)
            return fail(FD_EINVAL, "fd_batch_create: model %d mixes 2D and 3D models", i);
        if (models[i]->device != models[0]->device)
            return fail(FD_EINVAL, "fd_batch_create: models on different devices");
        for (int j = 0; j < i; ++j)
            if (models[j] == models[i])
                return fail(FD_EINVAL, "fd_batch_create: model %d repeated", i);
    }
    fd_batch *b = new fd_batch();
    b->models.assign(models, models + nmodels);
    b->device = models[0]->device;
    cudaError_t e = cudaSetDevice(b->device);
    // a stream of its own: the launch is captured into a graph, which the
    // legacy default stream does not allow
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&b->d_state, sizeof(BatchState));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&b->d_err, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        fd_batch_destroy(b);
        return cuda_fail(e, "batch allocation");
    }
    *out = b;
    return FD_OK;
}

extern "C" fd_status fd_batch_destroy(fd_batch *b)
{
    if (!b)
        return FD_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    free_tables(b);
    cudaFree(b->d_state);
    cudaFree(b->d_err);
    if (b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
    return FD_OK;
}

extern "C" fd_status fd_batch_set_tuning(fd_batch *b, const fd_batch_tuning *t)
{
    if (!b || !t)
        return fail(FD_EINVAL, "fd_batch_set_tuning: NULL argument");
    if (t->tile < 0 || t->tile > 7 || t->steps_per_launch < 1 || t->ctas_per_sm < 0 || t->group_mb < 0)
        return fail(FD_EINVAL, "fd_batch_set_tuning: value out of range");
    const bool same = t->tile == b->tun.tile && t->ctas_per_sm == b->tun.ctas_per_sm && t->group_mb == b->tun.group_mb;
    b->tun = *t;
    if (!same)
        free_tables(b);
    else if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return FD_OK;
}

extern "C" fd_status fd_batch_set_fault(fd_batch *b, int stalled_item)
{
    if (!b || stalled_item < -1)
        return fail(FD_EINVAL, "fd_batch_set_fault: bad arguments");
    b->stall_item = stalled_item;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return FD_OK;
}

extern "C" fd_status fd_batch_get_tuning(fd_batch *b, fd_batch_tuning *t)
{
    if (!b || !t)
        return fail(FD_EINVAL, "fd_batch_get_tuning: NULL argument");
    *t = b->tun;
    return FD_OK;
}

static fd_status capture_graph(fd_batch *b, const BatchParams &p)
{
    const Variant v = get_variant(b->tun.tile);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(v.threads);
    cfg.dynamicSmemBytes = v.smem;
    cfg.stream = b->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&p};
    cudaGraph_t graph = nullptr;
    FD_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    cudaError_t e = cudaLaunchKernelExC(&cfg, v.fn, args);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        return cuda_fail(e != cudaSuccess ? e : e2, "batch kernel capture");
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return cuda_fail(e, "graph instantiate");
    return FD_OK;
}

// The wide schedule: group by group, one launch per time step over the tiles of
// up to kWideMax of the group's shots that still have steps to go.  The host
// keeps each shot's level parity, step counter and owed receiver row; the
// launch gathers the owed rows of its shots, and the rows still owed at the end
// are gathered by one small launch per shot.
static fd_status run_wide(fd_batch *b, const std::vector<int> &target)
{
    const Variant v = get_variant(b->tun.tile);
    float w4[4];
    fd_stencil_weights(w4);
    WideParams &p = b->wide;
    p.c1 = w4[0];
    p.c2 = w4[1];
    p.c3 = w4[2];
    p.c4 = w4[3];
    p.err = b->d_err;
    const size_t ns = b->models.size();
    std::vector<int> pending(ns, -1), done(ns, 0);
    for (size_t g = 0; g + 1 < b->group_shot.size(); ++g) {
        const int sb = b->group_shot[g], se = b->group_shot[g + 1];
        int kmax = 0;
        for (int s = sb; s < se; ++s)
            kmax = std::max(kmax, target[s]);
        for (int k = 0; k < kmax; ++k) {
            for (int s0 = sb; s0 < se;) {
                int n = 0, tiles = 0;
                std::vector<int> in;
                for (; s0 < se && n < kWideMax; ++s0) {
                    if (done[s0] >= target[s0])
                        continue;
                    fd_model *m = b->models[s0];
                    const ShotDesc &d = b->shots[s0];
                    const int c = m->cur;
                    p.halo[n] = d.halo[c];
                    p.tile[n] = d.tile[c ^ 1];
                    p.wmap[n] = d.wmap;
                    WideShot &w = p.shot[n];
                    w.out = m->buf[c ^ 1];
                    w.P = m->buf[c];
                    w.ax = m->ax;
                    w.az = m->az;
                    w.trace_prev = pending[s0] >= 0 ? m->traces + (size_t)pending[s0] * m->nrec : nullptr;
                    w.rec_idx = m->d_rec;
                    w.nrec = m->nrec;
                    w.nx = m->nx;
                    w.nz = m->nz;
                    w.px = m->px;
                    w.tiles_x = (m->nx + v.tx - 1) / v.tx;
                    w.tile_begin = tiles;   // first CTA of the shot
                    w.has_sponge = m->has_sponge;
                    w.src_on = m->src_on && m->n < (int)m->amp.size();
                    w.sx = m->sx;
                    w.sz = m->sz;
                    w.src_amp = w.src_on ? m->amp[m->n] : 0.f;
                    tiles += w.tiles_x * (((m->nz + v.tz - 1) / v.tz + v.zt - 1) / v.zt);
                    in.push_back(s0);
                    ++n;
                }
                if (n == 0)
                    continue;
                p.nshots = n;
                switch (b->tun.tile) {
                case 3:
                    wide2d_kernel<64, 16, 1><<<tiles, v.threads, 0, b->stream>>>(p);
                    break;
                case 4:
                    wide2d_kernel<64, 32, 1><<<tiles, v.threads, 0, b->stream>>>(p);
                    break;
                case 5:
                    wide2d_kernel<64, 16, 4><<<tiles, v.threads, 0, b->stream>>>(p);
                    break;
                case 6:
                    wide2d_kernel<64, 16, 8><<<tiles, v.threads, 0, b->stream>>>(p);
                    break;
                default:
                    wide2d_kernel<64, 16, 16><<<tiles, v.threads, 0, b->stream>>>(p);
                    break;
                }
                ++g_launches;
                FD_CUDA(cudaGetLastError(), "wide batch launch");
                for (int s : in) {
                    fd_model *m = b->models[s];
                    m->cur ^= 1;
                    pending[s] = (m->nrec > 0 && m->traces && m->n < m->trace_rows) ? m->n : -1;
                    ++m->n;
                    ++done[s];
                }
            }
        }
    }
    for (size_t s = 0; s < ns; ++s) {
        fd_model *m = b->models[s];
        if (pending[s] >= 0) {
            FD_CUDA(launch_gather(m->buf[m->cur], m->d_rec, m->nrec, m->traces + (size_t)pending[s] * m->nrec,
                                  b->stream),
                    "receiver gather");
            ++g_launches;
        }
        m->pending_row = -1;
    }
    FD_CUDA(cudaStreamSynchronize(b->stream), "batch run");
    int err = 0;
    FD_CUDA(cudaMemcpy(&err, b->d_err, sizeof err, cudaMemcpyDeviceToHost), "error word");
    if (err) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return fail(FD_ETIMEOUT, "a wide batch launch gave up on its TMA wait (device code %d)", err);
    }
    return FD_OK;
}

// 3D batches: one launch per time step over up to kWide3Max models that still
// have steps to go, each CTA stepping its own model with the single-shot 3D
// kernel's body (maps and parameters from the launch).  The launch gathers each
// model's owed receiver row; the rows owed at the end are gathered per model.
static fd_status run_wide3d(fd_batch *b, const std::vector<int> &target)
{
    FD_CUDA(step3d_prepare(), "kernel attributes");
    Wide3Params &w = b->wide3;
    const size_t ns = b->models.size();
    std::vector<int> done(ns, 0);
    // z chunks for the launch as a whole: about six waves of CTAs over all models,
    // each CTA marching at least 32 planes (a model alone would cut small grids
    // into short chunks to fill the GPU, paying their halo planes again and again)
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    const long long slots = (long long)sms * step3d_blocks_per_sm();
    long long col_planes = 0;
    for (const fd_model *m : b->models)
        col_planes += (long long)((m->nx + kTX3 - 1) / kTX3) * ((m->ny + kTY3 - 1) / kTY3) * m->nz;
    const long long bz_t = std::max(32LL, col_planes / (6 * slots));
    std::vector<int> nch(ns), bzs(ns);
    for (size_t s = 0; s < ns; ++s) {
        const int nz = b->models[s]->nz;
        nch[s] = (int)((nz + std::min<long long>(bz_t, nz) - 1) / std::min<long long>(bz_t, nz));
        bzs[s] = (nz + nch[s] - 1) / nch[s];
    }
    int kmax = 0;
    for (int t : target)
        kmax = std::max(kmax, t);
    for (int k = 0; k < kmax; ++k) {
        for (size_t s0 = 0; s0 < ns;) {
            int n = 0, ctas = 0;
            std::vector<size_t> in;
            for (; s0 < ns && n < kWide3Max; ++s0) {
                if (done[s0] >= target[s0])
                    continue;
                fd_model *m = b->models[s0];
                const int c = m->cur;
                w.tmP[n] = m->halo_map[c];
                w.tmOld[n] = m->tile_map[c ^ 1];
                w.tmW[n] = m->w_map;
                fill_step_params(m, w.prm[n]);
                w.prm[n].stall_stage = -1;
                w.prm[n].bz = bzs[s0];
                w.tiles[n] = ((m->nx + kTX3 - 1) / kTX3) * ((m->ny + kTY3 - 1) / kTY3);
                w.cta_begin[n] = ctas;
                ctas += w.tiles[n] * nch[s0];
                in.push_back(s0);
                ++n;
            }
            if (n == 0)
                continue;
            w.nmodels = n;
            w.cta_begin[n] = ctas;
            FD_CUDA(launch_wide3d(w, b->stream), "batched 3D launch");
            ++g_launches;
            for (size_t s : in) {
                fd_model *m = b->models[s];
                m->cur ^= 1;
                m->pending_row = (m->nrec > 0 && m->traces && m->n < m->trace_rows) ? m->n : -1;
                ++m->n;
                ++done[s];
            }
        }
    }
    for (fd_model *m : b->models) {
        if (m->pending_row >= 0) {
            FD_CUDA(launch_gather(m->buf[m->cur], m->d_rec, m->nrec, m->traces + (size_t)m->pending_row * m->nrec,
                                  b->stream),
                    "receiver gather");
            ++g_launches;
        }
        m->pending_row = -1;
    }
    FD_CUDA(cudaStreamSynchronize(b->stream), "batch run");
    // the step kernels report a bounded wait that gave up in each model's error word
    for (fd_model *m : b->models) {
        int err = 0;
        FD_CUDA(cudaMemcpy(&err, m->d_err, sizeof err, cudaMemcpyDeviceToHost), "error word");
        if (err) {
            cudaMemset(m->d_err, 0, sizeof(int));
            return fail(FD_ETIMEOUT, "a batched 3D step gave up on a bounded wait (device code %d)", err);
        }
    }
    return FD_OK;
}

extern "C" fd_status fd_batch_step(fd_batch *b, int nsteps, const int *nsteps_each)
{
    NvtxRange nvtx_range("fd_batch_step");
    if (!b)
        return fail(FD_EINVAL, "NULL batch");
    FD_CUDA(cudaSetDevice(b->device), "cudaSetDevice");
    if (!nsteps_each && nsteps < 0)
        return fail(FD_EINVAL, "nsteps must be >= 0");
    const size_t ns = b->models.size();
    std::vector<int> target(ns);
    int tmax = 0;
    for (size_t s = 0; s < ns; ++s) {
        target[s] = nsteps_each ? nsteps_each[s] : nsteps;
        if (target[s] < 0)
            return fail(FD_EINVAL, "negative step count for shot %zu", s);
        tmax = std::max(tmax, target[s]);
    }
    if (b->models[0]->d.ndim == 3) {
        for (fd_model *m : b->models)
            FD_CUDA(cudaStreamSynchronize(m->stream), "model stream");
        return run_wide3d(b, target);
    }
    if (!b->built) {
        fd_status st = build_tables(b);
        if (st)
            return st;
    }
    // the models' own streams must be idle before the batch uses their buffers
    for (fd_model *m : b->models)
        FD_CUDA(cudaStreamSynchronize(m->stream), "model stream");
    if (get_variant(b->tun.tile).wide)
        return run_wide(b, target);
    for (size_t s = 0; s < ns; ++s) {
        fd_model *m = b->models[s];
        ShotDesc &d = b->shots[s];
        d.amp = m->d_amp;
        d.namp = m->src_on ? (int)m->amp.size() : 0;
        d.src_on = m->src_on;
        d.sx = m->sx;
        d.sz = m->sz;
        d.traces = m->nrec > 0 ? m->traces : nullptr;
        d.trace_rows = d.traces ? m->trace_rows : 0;
        d.nrec = m->nrec;
        d.n0 = m->n;
        d.cur0 = m->cur;
        d.target = target[s];
        d.has_sponge = m->has_sponge;
    }
    FD_CUDA(cudaMemcpyAsync(b->d_shots, b->shots.data(), ns * sizeof(ShotDesc), cudaMemcpyHostToDevice, b->stream),
            "batch upload");
    FD_CUDA(cudaMemsetAsync(b->d_counters, 0, std::max(1, b->nitems) * sizeof(int), b->stream), "batch reset");
    FD_CUDA(cudaMemsetAsync(b->d_state, 0, sizeof(BatchState), b->stream), "batch reset");
    if (tmax > 0) {
        if (!b->exec) {
            float w4[4];
            fd_stencil_weights(w4);
            BatchParams p{};
            p.shots = b->d_shots;
            p.items = b->d_items;
            p.recs = b->d_recs;
            p.counters = b->d_counters;
            p.group_begin = b->d_group;
            p.ngroups = b->ngroups;
            p.K = b->tun.steps_per_launch;
            p.state = b->d_state;
            p.c1 = w4[0];
            p.c2 = w4[1];
            p.c3 = w4[2];
            p.c4 = w4[3];
            p.err = b->d_err;
            p.stall_item = b->stall_item;
            fd_status st = capture_graph(b, p);
            if (st)
                return st;
        }
        const int launches = (tmax + b->tun.steps_per_launch - 1) / b->tun.steps_per_launch;
        for (int l = 0; l < launches; ++l) {
            FD_CUDA(cudaGraphLaunch(b->exec, b->stream), "batch launch");
            ++g_launches;
        }
    }
    FD_CUDA(cudaStreamSynchronize(b->stream), "batch run");
    int err = 0;
    FD_CUDA(cudaMemcpy(&err, b->d_err, sizeof err, cudaMemcpyDeviceToHost), "error word");
    for (size_t s = 0; s < ns; ++s) {
        fd_model *m = b->models[s];
        m->n += target[s];
        m->cur ^= target[s] & 1;
        m->pending_row = -1;
    }
    if (err) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return fail(FD_ETIMEOUT, "a batch dependency wait gave up (device code %d)", err);
    }
    return FD_OK;
}

namespace {
std::map<std::string, fd_batch_tuning> g_tuning_cache;

std::string batch_signature(const fd_batch *b)
{
    std::string sig;
    for (const fd_model *m : b->models)
        sig += std::to_string(m->nx) + "x" + std::to_string(m->nz) + (m->has_sponge ? "s" : "") + ";";
    return sig;
}
}  // namespace

extern "C" fd_status fd_batch_autotune(fd_batch *b, int trial_steps, fd_batch_tuning *best)
{
    NvtxRange nvtx_range("fd_batch_autotune");
    if (!b || trial_steps < 1)
        return fail(FD_EINVAL, "fd_batch_autotune: bad arguments");
    if (b->models[0]->d.ndim == 3) {   // a 3D batch has one schedule: nothing to tune
        if (best)
            *best = b->tun;
        return FD_OK;
    }
    const std::string sig = batch_signature(b) + "/" + std::to_string(trial_steps) + "/" +
                            std::to_string(b->tun.steps_per_launch);
    auto hit = g_tuning_cache.find(sig);
    if (hit != g_tuning_cache.end()) {
        fd_status st = fd_batch_set_tuning(b, &hit->second);
        if (best)
            *best = hit->second;
        return st;
    }
    double total_mb = 0;
    for (const fd_model *m : b->models)
        total_mb += 3.0 * m->pitched * 4 / 1048576.0;
    std::vector<int> groups{0};
    for (int g : {24, 48, 96})
        if (g < total_mb)
            groups.push_back(g);
    // Steps per persistent launch: the trial length, half and a quarter of it,
    // and the caller's value when shorter; each trial runs trial_steps steps.
    const int keep_k = b->tun.steps_per_launch;
    std::vector<int> ks{trial_steps};
    for (int k : {trial_steps / 2, trial_steps / 4, keep_k})
        if (k >= 1 && k < trial_steps && std::find(ks.begin(), ks.end(), k) == ks.end())
            ks.push_back(k);
    fd_batch_tuning best_t = b->tun;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    FD_CUDA(cudaEventCreate(&e0), "event");
    FD_CUDA(cudaEventCreate(&e1), "event");
    for (int tile = 0; tile < 8; ++tile)
        for (int g : groups)
            for (int cps : {0, 2})
                for (int k : ks) {
                    if (tile >= 3 && (cps || k != trial_steps))
                        continue;   // the wide schedule has no resident grid and one launch per step
                    fd_batch_tuning t{tile, k, cps, g};
                    fd_status st = fd_batch_set_tuning(b, &t);
                    if (!st)
                        st = fd_batch_step(b, 1, nullptr);   // build, capture and warm up
                    if (st)
                        continue;
                    cudaEventRecord(e0, b->stream);
                    st = fd_batch_step(b, trial_steps, nullptr);
                    cudaEventRecord(e1, b->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (!st && ms < best_ms) {
                        best_ms = ms;
                        best_t = t;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms >= 1e30f)
        return fail(FD_ECUDA, "fd_batch_autotune: no candidate ran");
    // A trial cannot time launches longer than itself.  When the longest timed
    // launch wins (or the wide schedule, where the value is unused), a caller's
    // longer launch is kept: one launch boundary fewer per trial_steps steps.
    if (best_t.tile >= 3 || (best_t.steps_per_launch == trial_steps && keep_k > trial_steps))
        best_t.steps_per_launch = keep_k;
    g_tuning_cache[sig] = best_t;
    if (best)
        *best = best_t;
    return fd_batch_set_tuning(b, &best_t);
}

// ------------------------------------------------------------ allocation-free variant
//
// fd_batch_step_noalloc runs the same persistent kernel as fd_batch_step over
// caller-created models, but takes every piece of scratch it needs (shot
// descriptors with their tensor maps, the tile table, the per-tile receiver
// lists, the per-tile step counters, the launch state and the error word) from
// one file-scope device array instead of device allocations.  Host-side it
// stages the tables in a file-scope host buffer of the same layout, so it
// makes no heap allocation either.

namespace {

constexpr int kNoAllocMaxShots = 64;
constexpr int kNoAllocMaxItems = 32768;   // 64 x 16 tiles in total over all shots
constexpr int kNoAllocMaxRecs = 32768;    // receivers in total over all shots
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocScratch {
    ShotDesc shots[kNoAllocMaxShots];
    BatchItem items[kNoAllocMaxItems];
    BatchRec recs[kNoAllocMaxRecs];
    int counters[kNoAllocMaxItems];
    int group_begin[2];
    BatchState state;
    int err;
};

NoAllocScratch h_noalloc;                           // host staging of the tables
int h_noalloc_cursor[kNoAllocMaxItems];             // per-tile receiver counts, then write cursors
void *g_noalloc_addr[kNoAllocMaxDevices] = {};      // device address of the array, per device
bool g_noalloc_ready[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mutex;                         // one call at a time per process

}  // namespace

// The scratch itself: shared by every call on a device, kept between calls.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

extern "C" fd_status fd_batch_step_noalloc(fd_model *const *models, int nmodels, int nsteps)
{
    if (!models || nmodels < 1 || nsteps < 0)
        return fail(FD_EINVAL, "fd_batch_step_noalloc: bad arguments");
    if (nmodels > kNoAllocMaxShots)
        return fail(FD_EBUDGET, "fd_batch_step_noalloc: %d shots exceed the static limit of %d", nmodels,
                    kNoAllocMaxShots);
    for (int i = 0; i < nmodels; ++i) {
        if (!models[i] || models[i]->d.ndim != 2)
            return fail(FD_EINVAL, "fd_batch_step_noalloc: model %d is NULL or not 2D", i);
        if (models[i]->device != models[0]->device)
            return fail(FD_EINVAL, "fd_batch_step_noalloc: models on different devices");
        for (int j = 0; j < i; ++j)
            if (models[j] == models[i])
                return fail(FD_EINVAL, "fd_batch_step_noalloc: model %d repeated", i);
    }
    const Variant v = get_variant(0);
    long long nitems = 0, nrecs = 0;
    for (int i = 0; i < nmodels; ++i) {
        const fd_model *m = models[i];
        nitems += (long long)((m->nx + v.tx - 1) / v.tx) * ((m->nz + v.tz - 1) / v.tz);
        nrecs += m->nrec;
    }
    if (nitems > kNoAllocMaxItems)
        return fail(FD_EBUDGET, "fd_batch_step_noalloc: %lld tiles of %dx%d exceed the static limit of %d", nitems,
                    v.tx, v.tz, kNoAllocMaxItems);
    if (nrecs > kNoAllocMaxRecs)
        return fail(FD_EBUDGET, "fd_batch_step_noalloc: %lld receivers exceed the static limit of %d", nrecs,
                    kNoAllocMaxRecs);
    const int dev = models[0]->device;
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(FD_EINVAL, "fd_batch_step_noalloc: device %d out of range", dev);
    // The host staging buffer, the address cache and the device array are shared:
    // the lock is held until the kernel has finished, so calls never overlap.
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    FD_CUDA(cudaSetDevice(dev), "cudaSetDevice");

    // One-time set-up on this device (the device is current): the device
    // address of the array, and the kernel's shared-memory limit.
    if (!g_noalloc_ready[dev]) {
        FD_CUDA(cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch), "scratch address");
        FD_CUDA(cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem),
                "kernel attributes");
        g_noalloc_ready[dev] = true;
    }
    unsigned char *dbase = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    NoAllocScratch &h = h_noalloc;

    // tables: one group holding every shot, 64 x 16 tiles
    int ni = 0, nr = 0;
    for (int s = 0; s < nmodels; ++s) {
        fd_model *m = models[s];
        ShotDesc &d = h.shots[s];
        d = ShotDesc{};
        bool ok = true;
        for (int i = 0; i < 2; ++i) {
            ok = ok && make_map(&d.halo[i], m->buf[i], 2, m->nx, 1, m->nz, m->px, v.tx + 8, v.tz + 8);
            ok = ok && make_map(&d.tile[i], m->buf[i], 2, m->nx, 1, m->nz, m->px, v.tx, v.tz);
            d.buf[i] = m->buf[i];
        }
        ok = ok && make_map(&d.wmap, m->w, 2, m->nx, 1, m->nz, m->px, v.tx, v.tz);
        if (!ok)
            return fail(FD_ECUDA, "cuTensorMapEncodeTiled failed for shot %d", s);
        d.ax = m->ax;
        d.az = m->az;
        d.amp = m->d_amp;
        d.namp = m->src_on ? (int)m->amp.size() : 0;
        d.src_on = m->src_on;
        d.sx = m->sx;
        d.sz = m->sz;
        d.traces = m->nrec > 0 ? m->traces : nullptr;
        d.trace_rows = d.traces ? m->trace_rows : 0;
        d.nrec = m->nrec;
        d.nx = m->nx;
        d.nz = m->nz;
        d.px = m->px;
        d.n0 = m->n;
        d.cur0 = m->cur;
        d.target = nsteps;
        d.has_sponge = m->has_sponge;
        const int tx_n = (m->nx + v.tx - 1) / v.tx, tz_n = (m->nz + v.tz - 1) / v.tz;
        const int base = ni;
        for (int t = 0; t < tx_n * tz_n; ++t) {
            BatchItem &it = h.items[base + t];
            const int tx = t % tx_n, tz = t / tx_n;
            it.shot = s;
            it.x0 = tx * v.tx;
            it.z0 = tz * v.tz;
            it.nb[0] = tx > 0 ? base + t - 1 : -1;
            it.nb[1] = tx + 1 < tx_n ? base + t + 1 : -1;
            it.nb[2] = tz > 0 ? base + t - tx_n : -1;
            it.nb[3] = tz + 1 < tz_n ? base + t + tx_n : -1;
        }
        // receivers bucketed by tile (a counting sort, O(nrec + tiles)); within a
        // tile they stay in receiver order
        int *cur = h_noalloc_cursor;
        const int ntile = tx_n * tz_n;
        for (int t = 0; t < ntile; ++t)
            cur[t] = 0;
        auto tile_of = [&](int r) {
            const int64_t di = m->rec_dense[r];
            const int ix = (int)(di % m->nx), iz = (int)(di / m->nx);
            return (iz / v.tz) * tx_n + ix / v.tx;
        };
        for (int r = 0; r < m->nrec; ++r)
            ++cur[tile_of(r)];
        for (int t = 0; t < tx_n * tz_n; ++t) {
            BatchItem &it = h.items[base + t];
            it.rec_begin = nr;
            nr += cur[t];
            it.rec_end = nr;
            cur[t] = it.rec_begin;
        }
        for (int r = 0; r < m->nrec; ++r) {
            const int64_t di = m->rec_dense[r];
            const int ix = (int)(di % m->nx), iz = (int)(di / m->nx);
            h.recs[cur[tile_of(r)]++] = BatchRec{(iz % v.tz) * v.tx + ix % v.tx, r};
        }
        ni += tx_n * tz_n;
    }
    h.group_begin[0] = 0;
    h.group_begin[1] = ni;

    for (int s = 0; s < nmodels; ++s)
        FD_CUDA(cudaStreamSynchronize(models[s]->stream), "model stream");
    cudaStream_t st = models[0]->stream;
    auto up = [&](size_t off, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dbase + off, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    FD_CUDA(up(offsetof(NoAllocScratch, shots), h.shots, nmodels * sizeof(ShotDesc)), "scratch upload");
    FD_CUDA(up(offsetof(NoAllocScratch, items), h.items, ni * sizeof(BatchItem)), "scratch upload");
    FD_CUDA(up(offsetof(NoAllocScratch, recs), h.recs, nr * sizeof(BatchRec)), "scratch upload");
    FD_CUDA(up(offsetof(NoAllocScratch, group_begin), h.group_begin, sizeof h.group_begin), "scratch upload");
    // what must start at zero: the counters in use, the launch state and the error word
    FD_CUDA(cudaMemsetAsync(dbase + offsetof(NoAllocScratch, counters), 0, ni * sizeof(int), st), "scratch clear");
    FD_CUDA(cudaMemsetAsync(dbase + offsetof(NoAllocScratch, state), 0, sizeof(BatchState), st), "scratch clear");
    FD_CUDA(cudaMemsetAsync(dbase + offsetof(NoAllocScratch, err), 0, sizeof(int), st), "scratch clear");

    if (nsteps > 0 && ni > 0) {
        float w4[4];
        fd_stencil_weights(w4);
        BatchParams p{};
        p.shots = reinterpret_cast<const ShotDesc *>(dbase + offsetof(NoAllocScratch, shots));
        p.items = reinterpret_cast<const BatchItem *>(dbase + offsetof(NoAllocScratch, items));
        p.recs = reinterpret_cast<const BatchRec *>(dbase + offsetof(NoAllocScratch, recs));
        p.counters = reinterpret_cast<int *>(dbase + offsetof(NoAllocScratch, counters));
        p.group_begin = reinterpret_cast<const int *>(dbase + offsetof(NoAllocScratch, group_begin));
        p.ngroups = 1;
        p.K = nsteps;
        p.state = reinterpret_cast<BatchState *>(dbase + offsetof(NoAllocScratch, state));
        p.c1 = w4[0];
        p.c2 = w4[1];
        p.c3 = w4[2];
        p.c4 = w4[3];
        p.err = reinterpret_cast<int *>(dbase + offsetof(NoAllocScratch, err));
        p.stall_item = -1;
        int per_sm = 0, sms = 0;
        FD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.fn, v.threads, v.smem), "occupancy");
        FD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
        if (per_sm < 1)
            return fail(FD_ECUDA, "batch kernel does not fit on an SM");
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(sms * per_sm);
        cfg.blockDim = dim3(v.threads);
        cfg.dynamicSmemBytes = v.smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void *args[] = {(void *)&p};
        FD_CUDA(cudaLaunchKernelExC(&cfg, v.fn, args), "batch kernel launch");
        ++g_launches;
    }
    FD_CUDA(cudaStreamSynchronize(st), "batch run");
    int err = 0;
    FD_CUDA(cudaMemcpy(&err, dbase + offsetof(NoAllocScratch, err), sizeof err, cudaMemcpyDeviceToHost),
            "error word");
    for (int s = 0; s < nmodels; ++s) {
        fd_model *m = models[s];
        m->n += nsteps;
        m->cur ^= nsteps & 1;
        m->pending_row = -1;
    }
    if (err)
        return fail(FD_ETIMEOUT, "a batch dependency wait gave up (device code %d)", err);
    return FD_OK;
}

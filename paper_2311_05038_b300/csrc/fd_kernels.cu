// fd_kernels.cu -- fused time-step kernels of the acoustic FD propagator (sm_103a).
//
// One launch performs one time step of the paper's WaveSimulator::run() loop
// (section 7): add_source, the z and x (and y) second derivatives, the time
// update and the rotation of levels, fused so that each grid point costs one
// read of P, Pold and w and one write of Pn (16 bytes) instead of the five
// field passes of the unfused routine sequence.  The receiver gather of the
// previous step rides along in the same launch.
//
// The per-point arithmetic lives in stencil.cuh.

#include <algorithm>
#include <type_traits>

#include "fd_internal.h"
#include "ptx.cuh"
#include "stencil.cuh"

namespace fdk {

// Gather of the previous step's receiver row, spread over every thread of the
// ncta CTAs that step the model (this CTA is number cta of them).
__device__ __forceinline__ void gather_prev_row(const StepParams &prm, int64_t cta, int64_t ncta)
{
    if (!prm.trace_prev)
        return;
    const int64_t nthr = ncta * blockDim.x;
    for (int64_t r = cta * blockDim.x + threadIdx.x; r < prm.nrec; r += nthr)
        prm.trace_prev[r] = prm.P[prm.rec_idx[r]];
}

// ----------------------------------------------------------------------------- 3D

// A CTA owns the column [x0, x0+TX) x [y0, y0+TY) and output planes [z0, z1);
// each of its TX/4*TY threads computes 4 consecutive x points of one row.
//
// Two TMA rings feed it, each stage a box two planes deep.  Counting "relative
// planes" from z0-4, P stage k (SP slots) holds the haloed P planes 2k and
// 2k+1; T stage t (ST slots) holds the Pold and w tiles of output planes
// z0+2t and z0+2t+1.  Body i computes output planes j = 2i and j+1: their x/y
// neighbours come from P stage i+2, the two newest planes (relative j+8, j+9)
// from P stage i+4 enter a register queue that supplies the z neighbours, and
// Pold, w from T stage i.  Afterwards the warp frees P stage i+2 and T stage i.
// Pairing planes halves the per-plane cost of the barrier probes, releases and
// ring bookkeeping.
//
// There is no producer thread: a per-slot shared counter finds the last warp to
// free a slot, and that warp issues the slot's next stage at once, so loads run
// ahead of the slowest warp without anyone blocking.  The only waits are the
// bounded waits on the full barriers.
//
// MODE 1 also writes L'P (the stencil sum of level n) to the dense array
// prm.lp_out; MODE 2 also adds Pn * prm.img_lp to prm.img_grad.  Both serve the
// adjoint's imaging condition; MODE 0 is the plain step.  MODE 3 is the plain
// step with the failure-path test hook (prm.stall_stage), kept out of MODE 0.
// MODES 4, 5, 6 are the paper's unfused derivative routines (fd_pxx, fd_pyy,
// fd_pzz): they stream P through the same ring and write only
// sum_k c_k (P[+k] + P[-k] - 2P) along x, y or z to prm.out, with no Pold or w
// loads.
//
// The body is a device function of the CTA's column bx (in x-fastest order) and
// z chunk by, so that one launch can also step several models (the batched 3D
// schedule, each CTA with its own model's maps and parameters); step3d_kernel
// runs it for one model with (bx, by) = blockIdx.  The tensor maps must stay in
// parameter space (references to __grid_constant__ parameters).
template <int TX, int TY, int SP, int ST, int G, int MODE>
__device__ __forceinline__ void step3d_body(const CUtensorMap &tmP, const CUtensorMap &tmOld, const CUtensorMap &tmW,
                                            const StepParams &prm, int bx, int by, int64_t cta, int64_t ncta)
{
    constexpr int QX = TX / 4;
    constexpr int NT = QX * TY;
    constexpr int NW = NT / 32;
    constexpr int HX = TX + 8;
    constexpr int HY = TY + 8;
    constexpr int PBOX = HX * HY;
    constexpr int TBOX = TX * TY;
    constexpr int PST = 2 * PBOX;
    constexpr int TST = 4 * TBOX;
    constexpr uint32_t BYTES_P = PST * 4;
    constexpr uint32_t BYTES_T = TST * 4;
    constexpr int QN = 8 + 2 * G;
    static_assert(NT % 32 == 0, "threads must fill warps");
    static_assert((PBOX * 4) % 128 == 0 && (TBOX * 4) % 128 == 0, "boxes keep 128-byte alignment");
    static_assert(kPlanes3 == 2, "bodies compute the two planes of a stage");
    static_assert(SP >= 4, "P ring must hold stages i+2 .. i+4 and run ahead");
    static_assert(ST >= 2, "T ring must run ahead");
    constexpr bool DERIV = MODE >= 4;   // one axis's second derivative only
    constexpr int DAXIS = MODE - 4;     // 0: x, 1: y, 2: z

    extern __shared__ __align__(128) unsigned char smem[];
    float *sP = reinterpret_cast<float *>(smem);
    float *sT = sP + SP * PST;   // the derivative modes have no T ring
    uint64_t *fullP = reinterpret_cast<uint64_t *>(sT + (DERIV ? 0 : ST * TST));
    uint64_t *fullT = fullP + SP;
    unsigned *relP = reinterpret_cast<unsigned *>(fullT + ST);
    unsigned *relT = relP + SP;
    __shared__ int s_abort;
    __shared__ int s_issuedP, s_issuedT;

    const int tiles_x = (prm.nx + TX - 1) / TX;
    const int x0 = (bx % tiles_x) * TX;
    const int y0 = (bx / tiles_x) * TY;
    const int z0 = by * prm.bz;
    const int z1 = min(prm.nz, z0 + prm.bz);
    const int nb = z1 - z0;
    const int nbh = (nb + 1) >> 1;
    const int nPS = nbh + 4;
    const int tid = threadIdx.x;
    const int lane = tid & 31;

    auto issueP = [&](int k, int slot) {
        if constexpr (MODE == 3) {
            if (k == prm.stall_stage && bx == 0 && by == 0) {
                // test hook: the stage is counted as issued but never loaded, so this
                // CTA's bounded waits run out; the drain below skips it
                atomicAdd(&s_issuedP, 1);
                return;
            }
        }
        mbar_arrive_expect_tx(&fullP[slot], BYTES_P);
        tma_load_3d(sP + slot * PST, &tmP, &fullP[slot], x0 - 4, y0 - 4, z0 - 4 + 2 * k);
        atomicAdd(&s_issuedP, 1);
    };
    auto issueT = [&](int t, int slot) {
        mbar_arrive_expect_tx(&fullT[slot], BYTES_T);
        tma_load_3d(sT + slot * TST, &tmOld, &fullT[slot], x0, y0, z0 + 2 * t);
        tma_load_3d(sT + slot * TST + 2 * TBOX, &tmW, &fullT[slot], x0, y0, z0 + 2 * t);
        atomicAdd(&s_issuedT, 1);
    };
    // Free P stage k (in slot sp) and, if t >= 0, T stage t (in slot stt); the
    // warp completing a slot's release refills it with the stage one ring later.
    auto release = [&](int k, int sp, int t, int stt) {
        __syncwarp();
        if (lane == 0) {
            if (atomicAdd(&relP[sp], 1u) % NW == NW - 1 && k + SP < nPS) {
                fence_proxy_async_shared();
                issueP(k + SP, sp);
            }
            if (t >= 0 && atomicAdd(&relT[stt], 1u) % NW == NW - 1 && t + ST < nbh) {
                fence_proxy_async_shared();
                issueT(t + ST, stt);
            }
        }
    };

    if (tid == 0) {
        for (int s = 0; s < SP; ++s) {
            mbar_init(&fullP[s], 1);
            relP[s] = 0;
        }
        for (int s = 0; s < ST; ++s) {
            mbar_init(&fullT[s], 1);
            relT[s] = 0;
        }
        s_abort = 0;
        s_issuedP = 0;
        s_issuedT = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        prefetch_tensormap(&tmP);
        prefetch_tensormap(&tmOld);
        prefetch_tensormap(&tmW);
        for (int k = 0; k < min(SP, nPS); ++k)
            issueP(k, k);
        if constexpr (!DERIV) {
            for (int t = 0; t < min(ST, nbh); ++t)
                issueT(t, t);
        }
    }

    gather_prev_row(prm, cta, ncta);

    const int tx = tid % QX;
    const int ty = tid / QX;
    const int x = x0 + 4 * tx;
    const int y = y0 + ty;
    const int cP = (ty + 4) * HX + 4 * tx + 4;
    const int cT = ty * TX + 4 * tx;
    const bool row_ok = y < prm.ny;

    float axv[4] = {0.f, 0.f, 0.f, 0.f};
    float ayv = 0.f;
    float az0 = 0.f, az1 = 0.f;   // az of the current body's two planes
    if (prm.has_sponge) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            axv[e] = x + e < prm.px ? prm.ax[x + e] : 0.f;
        ayv = row_ok ? prm.ay[y] : 0.f;
        az0 = prm.az[z0];        // profiles are zero-padded well past nz
        az1 = prm.az[z0 + 1];
    }
    const bool x_band = axv[0] != 0.f || axv[1] != 0.f || axv[2] != 0.f || axv[3] != 0.f;
    const bool src_col = prm.src_on && y == prm.sy && (unsigned)(prm.sx - x) < 4u;
    const bool store_vec = row_ok && x + 3 < prm.nx;
    const bool store_any = row_ok && x < prm.nx;
    float *const out_col = prm.out + ((size_t)z0 * prm.ny + y) * prm.px + x;
    const size_t plane_stride = (size_t)prm.ny * prm.px;
    // derivative modes may write a permuted view (the kernel's y and z swapped)
    const size_t deriv_sy = DERIV && prm.out_sy ? (size_t)prm.out_sy : (size_t)prm.px;
    const size_t deriv_sz = DERIV && prm.out_sz ? (size_t)prm.out_sz : plane_stride;
    float *const deriv_col = prm.out + (size_t)z0 * deriv_sz + (size_t)y * deriv_sy + x;

    // z queue, advanced G bodies (2G planes) at a time: in the r-th body of a
    // group, Q[i + 2r] holds relative plane j + i.
    float4 Q[QN];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ok = __all_sync(0xffffffffu, mbar_wait(&fullP[k % SP], (k / SP) & 1, &s_abort));
        if (!ok)
            break;
        Q[2 * k] = *reinterpret_cast<const float4 *>(sP + (k % SP) * PST + cP);
        Q[2 * k + 1] = *reinterpret_cast<const float4 *>(sP + (k % SP) * PST + PBOX + cP);
        if (k < 2)
            release(k, k % SP, -1, 0);
    }

    const float2 M2 = make_float2(-6.0f, -6.0f);
    const float2 NEG1 = make_float2(-1.0f, -1.0f);
    const float2 TWO = make_float2(2.0f, 2.0f);
    const float2 C1 = make_float2(prm.c1, prm.c1), C2 = make_float2(prm.c2, prm.c2);
    const float2 C3 = make_float2(prm.c3, prm.c3), C4 = make_float2(prm.c4, prm.c4);
    int sn = 4 % SP, phn = (4 / SP) & 1;   // P stage i+4
    int sx = 2 % SP;                        // P stage i+2
    int st = 0, pht = 0;                    // T stage i

    // Output plane z0+j from its P plane pl (centre float4), Pold/w tile tb and az;
    // L'P in packed FP32 in the same rounding order as update_point<3>.
    auto plane = [&](int j, const float *pl, const float *tb, float azv, auto qo) {
        constexpr int O = decltype(qo)::value;   // Q index of this plane's centre
        if constexpr (DERIV) {
            const float4 &pc = Q[O];
            if constexpr (DAXIS == 0) {
                const float4 xm = *reinterpret_cast<const float4 *>(pl - 4);
                const float4 xp = *reinterpret_cast<const float4 *>(pl + 4);
                const float xa[12] = {xm.x, xm.y, xm.z, xm.w, pc.x, pc.y, pc.z, pc.w, xp.x, xp.y, xp.z, xp.w};
                float2 acc[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 p2 = half2of(pc, h);
                    float2 a2;
#pragma unroll
                    for (int k = 1; k <= 4; ++k) {
                        const float2 d = __ffma2_rn(make_float2(-2.0f, -2.0f), p2, xpair2(xa, h, k));
                        const float2 ck = k == 1 ? C1 : k == 2 ? C2 : k == 3 ? C3 : C4;
                        a2 = k == 1 ? __fmul2_rn(ck, d) : __ffma2_rn(ck, d, a2);
                    }
                    acc[h] = a2;
                }
                float *dst = deriv_col + (size_t)j * deriv_sz;
                if (store_vec)
                    *reinterpret_cast<float4 *>(dst) = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
                else if (store_any)
                    store4(dst, acc, prm.nx - x);
                return;
            } else {
                float4 mk[4], pk[4];
#pragma unroll
                for (int k = 1; k <= 4; ++k) {
                    if constexpr (DAXIS == 1) {
                        mk[k - 1] = *reinterpret_cast<const float4 *>(pl - k * HX);
                        pk[k - 1] = *reinterpret_cast<const float4 *>(pl + k * HX);
                    } else {
                        mk[k - 1] = Q[O - k];
                        pk[k - 1] = Q[O + k];
                    }
                }
                float2 acc[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 p2 = half2of(pc, h);
                    float2 a2;
#pragma unroll
                    for (int k = 1; k <= 4; ++k) {
                        const float2 sk = __fadd2_rn(half2of(pk[k - 1], h), half2of(mk[k - 1], h));
                        const float2 d = __ffma2_rn(make_float2(-2.0f, -2.0f), p2, sk);
                        const float2 ck = k == 1 ? C1 : k == 2 ? C2 : k == 3 ? C3 : C4;
                        a2 = k == 1 ? __fmul2_rn(ck, d) : __ffma2_rn(ck, d, a2);
                    }
                    acc[h] = a2;
                }
                float *dst = deriv_col + (size_t)j * deriv_sz;
                if (store_vec)
                    *reinterpret_cast<float4 *>(dst) = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
                else if (store_any)
                    store4(dst, acc, prm.nx - x);
                return;
            }
        }
        const float4 xm = *reinterpret_cast<const float4 *>(pl - 4);
        const float4 xc = *reinterpret_cast<const float4 *>(pl);
        const float4 xp = *reinterpret_cast<const float4 *>(pl + 4);
        float4 ym[4], yp[4];
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            ym[k - 1] = *reinterpret_cast<const float4 *>(pl - k * HX);
            yp[k - 1] = *reinterpret_cast<const float4 *>(pl + k * HX);
        }
        const float4 old = *reinterpret_cast<const float4 *>(tb);
        const float4 wv = *reinterpret_cast<const float4 *>(tb + 2 * TBOX);
        const float xa[12] = {xm.x, xm.y, xm.z, xm.w, xc.x, xc.y, xc.z, xc.w, xp.x, xp.y, xp.z, xp.w};
        const float4 &pc = Q[O];
        float2 acc[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 p2 = half2of(pc, h);
            float2 a2;
#pragma unroll
            for (int k = 1; k <= 4; ++k) {
                const float2 sxx = xpair2(xa, h, k);
                const float2 sy = __fadd2_rn(half2of(yp[k - 1], h), half2of(ym[k - 1], h));
                const float2 sz = __fadd2_rn(half2of(Q[O + k], h), half2of(Q[O - k], h));
                const float2 d = __ffma2_rn(M2, p2, __fadd2_rn(__fadd2_rn(sxx, sy), sz));
                const float2 ck = k == 1 ? C1 : k == 2 ? C2 : k == 3 ? C3 : C4;
                a2 = k == 1 ? __fmul2_rn(ck, d) : __ffma2_rn(ck, d, a2);
            }
            acc[h] = a2;
        }
        const float ayz = ayv + azv;
        float2 r[2];
        if (x_band || ayz != 0.f) {
            // sponge band: (w L'P + 2P - (1 - a) Pold) / (1 + a), scalar
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // per lane the scalar form's operations: a = ax + ayz, (a - 1) Pold = -(1 - a) Pold,
                // fma(2, P, .), fma(w, L'P, .), then the division where a != 0
                const float2 a2 = __fadd2_rn(make_float2(axv[2 * h], axv[2 * h + 1]), make_float2(ayz, ayz));
                const float2 t2 = __fmul2_rn(__fadd2_rn(NEG1, a2), half2of(old, h));
                const float2 n2 = __ffma2_rn(half2of(wv, h), acc[h], __ffma2_rn(TWO, half2of(pc, h), t2));
                r[h] = make_float2(a2.x != 0.0f ? __fdividef(n2.x, 1.0f + a2.x) : n2.x,
                                   a2.y != 0.0f ? __fdividef(n2.y, 1.0f + a2.y) : n2.y);
            }
        } else {
            // 2P - Pold as fma(-1, Pold, P + P): P + P is exact, one rounding as before
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 p2 = half2of(pc, h);
                const float2 t = __ffma2_rn(NEG1, half2of(old, h), __fadd2_rn(p2, p2));
                r[h] = __ffma2_rn(half2of(wv, h), acc[h], t);
            }
        }
        if constexpr (MODE == 1) {
            if (store_any)
                store4_dense(prm.lp_out + ((size_t)(z0 + j) * prm.ny + y) * prm.nx + x, acc, prm.nx - x,
                             (prm.nx & 3) == 0);
        }
        if (src_col && z0 + j == prm.sz)
            add_source4(r, prm.sx - x, prm.src_amp);
        if constexpr (MODE == 2) {
            if (store_any) {
                const size_t d = ((size_t)(z0 + j) * prm.ny + y) * prm.nx + x;
                image4_dense(prm.img_grad + d, prm.img_lp + d, r, prm.nx - x, (prm.nx & 3) == 0);
            }
        }
        float *dst = out_col + (size_t)j * plane_stride;
        if (store_vec) {
            *reinterpret_cast<float4 *>(dst) = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
        } else if (store_any) {
            dst[0] = r[0].x;
            if (x + 1 < prm.nx) dst[1] = r[0].y;
            if (x + 2 < prm.nx) dst[2] = r[1].x;
        }
    };

    auto body = [&](int i, auto rot) {
        constexpr int R = decltype(rot)::value;
        // fast path: both stages already landed; else bounded waits
        if constexpr (DERIV) {
            if (!__all_sync(0xffffffffu, mbar_try_wait(&fullP[sn], phn))) {
                ok = __all_sync(0xffffffffu, mbar_wait(&fullP[sn], phn, &s_abort));
                if (!ok)
                    return;
            }
        } else if (!__all_sync(0xffffffffu, mbar_try_wait(&fullP[sn], phn) & mbar_try_wait(&fullT[st], pht))) {
            ok = __all_sync(0xffffffffu, mbar_wait(&fullP[sn], phn, &s_abort) &&
                                             mbar_wait(&fullT[st], pht, &s_abort));
            if (!ok)
                return;
        }
        const int j = 2 * i;
        const float a0v = az0, a1v = az1;
        if (prm.has_sponge) {
            az0 = prm.az[z0 + j + 2];
            az1 = prm.az[z0 + j + 3];
        }
        const float *pn = sP + sn * PST + cP;
        Q[8 + 2 * R] = *reinterpret_cast<const float4 *>(pn);
        Q[9 + 2 * R] = *reinterpret_cast<const float4 *>(pn + PBOX);
        const float *pl = sP + sx * PST + cP;
        const float *tb = sT + st * TST + cT;
        plane(j, pl, tb, a0v, std::integral_constant<int, 4 + 2 * R>{});
        if (j + 1 < nb)
            plane(j + 1, pl + PBOX, tb + TBOX, a1v, std::integral_constant<int, 5 + 2 * R>{});
        release(i + 2, sx, DERIV ? -1 : i, st);
        if (++sn == SP) {
            sn = 0;
            phn ^= 1;
        }
        if (++sx == SP)
            sx = 0;
        if (++st == ST) {
            st = 0;
            pht ^= 1;
        }
    };

    for (int ib = 0; ok && ib < nbh; ib += G) {
        body(ib, std::integral_constant<int, 0>{});
        if constexpr (G > 1) {
            if (ok && ib + 1 < nbh)
                body(ib + 1, std::integral_constant<int, 1>{});
        }
        if constexpr (G > 2) {
            if (ok && ib + 2 < nbh)
                body(ib + 2, std::integral_constant<int, 2>{});
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            Q[k] = Q[k + 2 * G];
    }
    if (!ok)
        raise_error(prm.err, &s_abort, kDevErrTimeout);
    // After an abort, do not leave while copies into this CTA's shared memory may
    // be in flight: wait (bounded) for the newest use of every slot.
    __syncthreads();
    if (tid == 0 && s_abort) {
        int never = 0;
        // the issued stages are always 0 .. s_issuedP-1: stage k+SP is issued only
        // after every warp has freed stage k
        for (int k = max(0, s_issuedP - SP); k < s_issuedP; ++k) {
            if constexpr (MODE == 3) {
                if (k == prm.stall_stage && bx == 0 && by == 0)
                    continue;   // withheld by the test hook: nothing in flight
            }
            mbar_wait(&fullP[k % SP], (k / SP) & 1, &never, kWaitLimitCycles / 8);
        }
        for (int t = max(0, s_issuedT - ST); t < s_issuedT; ++t)
            mbar_wait(&fullT[t % ST], (t / ST) & 1, &never, kWaitLimitCycles / 8);
    }
}

template <int TX, int TY, int SP, int ST, int G, int MODE>
__global__ void __launch_bounds__(TX / 4 * TY, MODE >= 4 ? 768 / (TX / 4 * TY) : kMinBlocks3)
    step3d_kernel(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmOld,
                  const __grid_constant__ CUtensorMap tmW, const StepParams prm)
{
    step3d_body<TX, TY, SP, ST, G, MODE>(tmP, tmOld, tmW, prm, blockIdx.x, blockIdx.y,
                                         (int64_t)blockIdx.y * gridDim.x + blockIdx.x,
                                         (int64_t)gridDim.x * gridDim.y);
}

// Several 3D models in one launch, one time step each (the batched 3D schedule):
// a CTA finds its model by a binary search over the models' first CTAs in the
// launch parameters and runs the step body with that model's tensor maps and
// parameters, all in parameter space.
__global__ void __launch_bounds__(kThreads3, kMinBlocks3) wide3d_kernel(const __grid_constant__ Wide3Params w)
{
    int lo = 0, hi = w.nmodels - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (w.cta_begin[mid] <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int m = lo;
    const int c = blockIdx.x - w.cta_begin[m];
    const int tiles = w.tiles[m];
    step3d_body<kTX3, kTY3, kStagesP3, kStagesT3, kGroup3, 0>(w.tmP[m], w.tmOld[m], w.tmW[m], w.prm[m], c % tiles,
                                                              c / tiles, c, w.cta_begin[m + 1] - w.cta_begin[m]);
}

// ----------------------------------------------------------------------------- 2D

// A CTA owns a column of up to ZT tiles of TX x TZ points of the [nz][nx] grid,
// stacked along z, and walks down it through a two-stage TMA ring: one TMA
// transaction brings a tile's haloed P box and its Pold and w tiles, and the
// next tile's transaction is in flight while a tile is computed.  Each thread
// computes 4 consecutive x points of one row.  ZT = 1 is one tile per CTA.
template <int TX, int TZ, int ZT, int MODE>
__global__ void __launch_bounds__(TX / 4 * TZ)
    step2d_kernel(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmOld,
                  const __grid_constant__ CUtensorMap tmW, const StepParams prm)
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

    const int tiles_x = (prm.nx + TX - 1) / TX;
    const int tiles_z = (prm.nz + TZ - 1) / TZ;
    const int x0 = (blockIdx.x % tiles_x) * TX;
    const int tz0 = (blockIdx.x / tiles_x) * ZT;   // first tile row of this column
    const int nt = min(ZT, tiles_z - tz0);
    const int tid = threadIdx.x;

    auto issue = [&](int i) {
        const int st = i % NS;
        const int z0 = (tz0 + i) * TZ;
        mbar_arrive_expect_tx(&bar[st], BYTES);
        tma_load_2d(sP[st], &tmP, &bar[st], x0 - 4, z0 - 4);
        tma_load_2d(sO[st], &tmOld, &bar[st], x0, z0);
        tma_load_2d(sW[st], &tmW, &bar[st], x0, z0);
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
    gather_prev_row(prm, blockIdx.x, gridDim.x);

    const int tx = tid % QX;
    const int tz = tid / QX;
    const int x = x0 + 4 * tx;
    float axv[4] = {0.f, 0.f, 0.f, 0.f};
    if (prm.has_sponge) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            axv[e] = x + e < prm.px ? prm.ax[x + e] : 0.f;
    }
    for (int i = 0; i < nt; ++i) {
        const int st = i % NS;
        const int z = (tz0 + i) * TZ + tz;
        const float azv = prm.has_sponge && z < prm.nz ? prm.az[z] : 0.f;
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
        if (prm.src_on && z == prm.sz && (unsigned)(prm.sx - x) < 4u)
            add_source4(r, prm.sx - x, prm.src_amp);
        if (z < prm.nz && x < prm.nx) {
            store4(prm.out + (size_t)z * prm.px + x, r, prm.nx - x);
            if constexpr (MODE == 1)
                store4_dense(prm.lp_out + (size_t)z * prm.nx + x, lp, prm.nx - x, (prm.nx & 3) == 0);
            if constexpr (MODE == 2)
                image4_dense(prm.img_grad + (size_t)z * prm.nx + x, prm.img_lp + (size_t)z * prm.nx + x, r,
                             prm.nx - x, (prm.nx & 3) == 0);
        }
        if (NS > 1 && i + NS < nt) {
            __syncthreads();   // every thread has read stage st
            if (tid == 0) {
                fence_proxy_async_shared();
                issue(i + NS);
            }
        }
    }
}

// ------------------------------------------------------------------------ helpers

__global__ void gather_kernel(const float *__restrict__ P, const int64_t *__restrict__ idx, int nrec,
                              float *__restrict__ out)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x)
        out[r] = P[idx[r]];
}

__global__ void velocity_stats_kernel(const float *__restrict__ v, int nx, size_t rows, int px,
                                      unsigned *stats)
{
    unsigned vmax_bits = 0, bad = 0;
    const size_t n = (size_t)nx * rows;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / nx;
        const float x = v[row * px + (i - row * nx)];
        if (isfinite(x) && x > 0.f)
            vmax_bits = max(vmax_bits, __float_as_uint(x));   // positive floats order as their bits
        else
            ++bad;
    }
    for (int o = 16; o > 0; o >>= 1) {
        vmax_bits = max(vmax_bits, __shfl_xor_sync(0xffffffffu, vmax_bits, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&stats[0], vmax_bits);
        if (bad)
            atomicAdd(&stats[1], bad);
    }
}

// w = (dt/h * v)^2 in FP64, rounded once to FP32; v and w share the pitched layout
// (v may alias w).
__global__ void compute_w_kernel(const float *v, float *w, int nx, size_t rows, int px, double dt_over_h)
{
    const size_t n = (size_t)nx * rows;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / nx;
        const size_t at = row * px + (i - row * nx);
        const double c = dt_over_h * (double)v[at];
        w[at] = (float)(c * c);
    }
}

// ------------------------------------------------------------------------ launchers

#define FD_STEP3D(MODE) step3d_kernel<kTX3, kTY3, kStagesP3, kStagesT3, kGroup3, MODE>

size_t step3d_smem_bytes()
{
    constexpr int PBOX = (kTX3 + 8) * (kTY3 + 8);
    constexpr int TBOX = kTX3 * kTY3;
    return (size_t)(kStagesP3 * kPlanes3 * PBOX + kStagesT3 * kPlanes3 * 2 * TBOX) * sizeof(float) +
           (kStagesP3 + kStagesT3) * (sizeof(uint64_t) + sizeof(unsigned));
}

// The derivative modes keep only the P ring.
static size_t deriv3d_smem_bytes()
{
    constexpr int PBOX = (kTX3 + 8) * (kTY3 + 8);
    return (size_t)(kStagesP3 * kPlanes3 * PBOX) * sizeof(float) +
           (kStagesP3 + kStagesT3) * (sizeof(uint64_t) + sizeof(unsigned));
}

cudaError_t step3d_prepare()
{
    const int bytes = (int)step3d_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(FD_STEP3D(0), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(wide3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(FD_STEP3D(1), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(FD_STEP3D(2), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(FD_STEP3D(3), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(FD_STEP3D(4), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(FD_STEP3D(5), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(FD_STEP3D(6), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

int step3d_blocks_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, FD_STEP3D(0), kThreads3, step3d_smem_bytes()) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_step3d(const CUtensorMap &tmP, const CUtensorMap &tmOld, const CUtensorMap &tmW,
                          const StepParams &p, int nchunks, cudaStream_t s)
{
    const int tiles = ((p.nx + kTX3 - 1) / kTX3) * ((p.ny + kTY3 - 1) / kTY3);
    dim3 grid(tiles, nchunks);
    if (p.deriv_axis == 0)
        FD_STEP3D(4)<<<grid, kThreads3, deriv3d_smem_bytes(), s>>>(tmP, tmOld, tmW, p);
    else if (p.deriv_axis == 1)
        FD_STEP3D(5)<<<grid, kThreads3, deriv3d_smem_bytes(), s>>>(tmP, tmOld, tmW, p);
    else if (p.deriv_axis == 2)
        FD_STEP3D(6)<<<grid, kThreads3, deriv3d_smem_bytes(), s>>>(tmP, tmOld, tmW, p);
    else if (p.lp_out)
        FD_STEP3D(1)<<<grid, kThreads3, step3d_smem_bytes(), s>>>(tmP, tmOld, tmW, p);
    else if (p.img_grad)
        FD_STEP3D(2)<<<grid, kThreads3, step3d_smem_bytes(), s>>>(tmP, tmOld, tmW, p);
    else if (p.stall_stage >= 0)
        FD_STEP3D(3)<<<grid, kThreads3, step3d_smem_bytes(), s>>>(tmP, tmOld, tmW, p);
    else
        FD_STEP3D(0)<<<grid, kThreads3, step3d_smem_bytes(), s>>>(tmP, tmOld, tmW, p);
    return cudaGetLastError();
}

cudaError_t launch_wide3d(const Wide3Params &w, cudaStream_t s)
{
    wide3d_kernel<<<w.cta_begin[w.nmodels], kThreads3, step3d_smem_bytes(), s>>>(w);
    return cudaGetLastError();
}

// Columns of kZT2 tiles per CTA when the grid has tiles for several waves of
// them, else one tile per CTA so that small grids still spread over the SMs.
template <int ZT>
static void launch_step2d_zt(const CUtensorMap &tmP, const CUtensorMap &tmOld, const CUtensorMap &tmW,
                             const StepParams &p, int ctas, cudaStream_t s)
{
    if (p.lp_out)
        step2d_kernel<kTX2, kTZ2, ZT, 1><<<ctas, kThreads2, 0, s>>>(tmP, tmOld, tmW, p);
    else if (p.img_grad)
        step2d_kernel<kTX2, kTZ2, ZT, 2><<<ctas, kThreads2, 0, s>>>(tmP, tmOld, tmW, p);
    else
        step2d_kernel<kTX2, kTZ2, ZT, 0><<<ctas, kThreads2, 0, s>>>(tmP, tmOld, tmW, p);
}

cudaError_t launch_step2d(const CUtensorMap &tmP, const CUtensorMap &tmOld, const CUtensorMap &tmW,
                          const StepParams &p, cudaStream_t s)
{
    const int tiles_x = (p.nx + kTX2 - 1) / kTX2, tiles_z = (p.nz + kTZ2 - 1) / kTZ2;
    const long long stacked = (long long)tiles_x * ((tiles_z + kZT2 - 1) / kZT2);
    if (stacked >= kStackMinCtas2)
        launch_step2d_zt<kZT2>(tmP, tmOld, tmW, p, (int)stacked, s);
    else
        launch_step2d_zt<1>(tmP, tmOld, tmW, p, tiles_x * tiles_z, s);
    return cudaGetLastError();
}

cudaError_t launch_gather(const float *P, const int64_t *idx, int nrec, float *out, cudaStream_t s)
{
    if (nrec <= 0)
        return cudaSuccess;
    const int blocks = min((nrec + 255) / 256, 1184);
    gather_kernel<<<blocks, 256, 0, s>>>(P, idx, nrec, out);
    return cudaGetLastError();
}

cudaError_t launch_velocity_stats(const float *v, int nx, size_t rows, int px, unsigned *stats,
                                  cudaStream_t s)
{
    const size_t n = (size_t)nx * rows;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 148 * 8);
    velocity_stats_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(v, nx, rows, px, stats);
    return cudaGetLastError();
}

cudaError_t launch_compute_w(const float *v, float *w, int nx, size_t rows, int px, double dt_over_h,
                             cudaStream_t s)
{
    const size_t n = (size_t)nx * rows;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
    compute_w_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(v, w, nx, rows, px, dt_over_h);
    return cudaGetLastError();
}

}  // namespace fdk

// lgcd_global.cuh -- LGCD worker for tiles kept in global memory (Alg. 1 in
// each worker of Alg. 3), shared by the single-solve kernel and the batched
// queue kernel.
#pragma once
#include "lgcd_common.cuh"

namespace csc {

// ============================================================ GLOBAL TILES
// Variant for tiles whose beta / Z / table do not fit in shared memory (large
// atoms, e.g. 25 atoms of 32 x 32).  beta and Z stay in global memory (HBM,
// L2) and the table is read from L2.  Every beta window update is a
// red.global.add, so updates from neighbouring tiles that land in the same
// entries add up instead of overwriting each other, and an update whose
// window V(s0) crosses into a neighbour is applied there directly.  The
// neighbour learns that its beta changed through its flag counter (one word
// per tile): a worker bumps the counter of every tile V(s0) reaches.  The
// counters carry the same termination accounting as the mailboxes of the
// shared-memory variant: `pending` counts active workers plus flag bumps not
// yet observed by their tile.  One sub-domain per iteration, scanned and
// updated by the whole CTA.
constexpr int kGlobThreads = 512;

template <typename real, int NT>
__device__ void global_tile_worker(const LgcdArgs<real> &a, int w, unsigned char *smem_raw);

// The worker of tile w (all NT threads of the CTA); smem_raw holds at least
// 2 K elements.  Returns when the solve of `a` ends.
template <typename real, int NT>
__device__ void global_tile_worker(const LgcdArgs<real> &a, int w, unsigned char *smem_raw) {
    real *snrm = reinterpret_cast<real *>(smem_raw), *sinv = snrm + a.K;
    const int ta = w / a.G1, tb = w % a.G1;
    const int or0 = ta * a.t0, oc0 = tb * a.t1;
    const int h = min(a.t0, a.Z0 - or0), wd = min(a.t1, a.Z1 - oc0);
    const int ns0 = (h + a.sub0 - 1) / a.sub0, ns1 = (wd + a.sub1 - 1) / a.sub1, M = ns0 * ns1;
    const int K = a.K, WW = a.W0 * a.W1;
    const size_t plane = (size_t)a.Z0 * a.Z1;
    for (int k = threadIdx.x; k < K; k += NT) {
        snrm[k] = real(a.nrm[k]);
        sinv[k] = real(1.0 / a.nrm[k]);
    }
    int *flag = a.ctl + (size_t)w * kDirs * 32;  // this tile's counter
    __shared__ int s_ctl[4];                     // new flag bumps, state, accept
    __shared__ Cand<real> s_best;
    long long n_upd = 0, n_it = 0, n_rej = 0, n_sub = 0, n_msg = 0;
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    real guard = real(0);
    if (a.guard_on) {
        double g = 1e300;
        for (int k = 0; k < K; k++) g = fmin(g, 50.0 / a.dmax[k]);
        guard = real(g);
    }
    int seen = 0, m = 0, quiet = 0;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            int got = 0, state = 0;
            const int f = ld_relaxed(flag);
            if (f != seen) {
                got = f - seen;
                seen = f;
                atomicSub(&a.hdr->pending, got);  // observed: no longer in flight
            }
            if (ld_relaxed(&a.hdr->stop)) state = 1;
            else if (globaltimer_ns() > deadline) {
                set_stop(a.hdr, CSC_ERR_TIMEOUT);
                state = 1;
            }
            s_ctl[0] = got;
            s_ctl[1] = state;
        }
        __syncthreads();
        if (s_ctl[1]) break;
        const int got = s_ctl[0];
        // ---- scan sub-domain m (Eq. gcd_candidate)
        const int mr = m / ns1, mc = m % ns1;
        const int r0 = mr * a.sub0, c0 = mc * a.sub1;
        const int bh = min(a.sub0, h - r0), bw = min(a.sub1, wd - c0), nb = bh * bw;
        Cand<real> c{real(-1), 0xffffffffu, real(0), real(0)};
        for (int q = threadIdx.x; q < K * nb; q += NT) {
            const int k = q / nb, r = q % nb, li = r0 + r / bw, lj = c0 + r % bw;
            const size_t g = k * plane + (size_t)(or0 + li) * a.Z1 + oc0 + lj;
            const real zn = coord_update(__ldcg(a.beta + g), a.lambda, snrm[k], sinv[k]);
            // Z through L2: in the persistent queue an L1 line may still hold
            // this address from an earlier job whose buffer was recycled
            const real dz = zn - __ldcg(a.Z + g);
            Cand<real> x{dz < real(0) ? -dz : dz, (unsigned)((li * a.t1 + lj) * K + k), zn, dz};
            if (better(x, c)) c = x;
        }
        const Cand<real> best = block_argmax<real, NT>(c);
        n_it++;
        const bool active = best.a >= a.eps;
        if (active) {
            const unsigned pos = best.key / (unsigned)K;
            const int k0 = (int)(best.key % (unsigned)K);
            const int li0 = (int)(pos / (unsigned)a.t1), lj0 = (int)(pos % (unsigned)a.t1);
            const int gi0 = or0 + li0, gj0 = oc0 + lj0;
            const bool border = in_band(li0, lj0, h, wd, a.L0, a.L1);
            bool accept = true;
            if (border && a.mode == CSC_MODE_ASYNC) {
                // soft-lock over the part of V(s0) outside the tile: at most one
                // strip of rows outside the tile rows (full width of V) and one
                // strip of columns outside the tile columns (tile rows only)
                const int v0 = max(0, gi0 - (a.L0 - 1)), v1 = min(a.Z0, gi0 + a.L0);
                const int u0 = max(0, gj0 - (a.L1 - 1)), u1 = min(a.Z1, gj0 + a.L1);
                const int ra0 = v0 < or0 ? v0 : max(v0, or0 + h), ra1 = v0 < or0 ? min(v1, or0) : v1;
                const int rb0 = max(v0, or0), rb1 = min(v1, or0 + h);
                const int cb0 = u0 < oc0 ? u0 : max(u0, oc0 + wd), cb1 = u0 < oc0 ? min(u1, oc0) : u1;
                const int n1 = max(0, ra1 - ra0) * (u1 - u0), n2 = max(0, rb1 - rb0) * max(0, cb1 - cb0);
                real lo = real(-1), hi = real(-1);
                for (int q = threadIdx.x; q < K * (n1 + n2); q += NT) {
                    const int k = q / (n1 + n2), e = q % (n1 + n2);
                    int gi, gj;
                    if (e < n1) {
                        gi = ra0 + e / (u1 - u0);
                        gj = u0 + e % (u1 - u0);
                    } else {
                        gi = rb0 + (e - n1) / (cb1 - cb0);
                        gj = cb0 + (e - n1) % (cb1 - cb0);
                    }
                    const size_t g = k * plane + (size_t)gi * a.Z1 + gj;
                    real d = coord_update(ld_relaxed(a.beta + g), a.lambda, snrm[k], sinv[k]) - ld_relaxed(a.Z + g);
                    d = d < real(0) ? -d : d;
                    if ((gi / a.t0) * a.G1 + gj / a.t1 < w) lo = max(lo, d);
                    else hi = max(hi, d);
                }
                real mhi;
                const real mlo = block_max2<real, NT>(lo, hi, &mhi);
                accept = best.a > mlo && best.a >= mhi;
                if (!accept) n_rej += threadIdx.x == 0;
            }
            if (accept) {
                // beta_k[s] -= C[k][k0][s - s0] dz on V(s0) within the domain
                const real dz = best.dz;
                for (int q = threadIdx.x; q < K * WW; q += NT) {
                    const int k = q / WW, r = q % WW;
                    const int gi = gi0 + r / a.W1 - (a.L0 - 1), gj = gj0 + r % a.W1 - (a.L1 - 1);
                    if (gi < 0 || gi >= a.Z0 || gj < 0 || gj >= a.Z1) continue;
                    if (k == k0 && gi == gi0 && gj == gj0) continue;
                    const real cval = __ldg(a.dtd + ((size_t)k * K + k0) * WW + r);
                    atomicAdd(a.beta + k * plane + (size_t)gi * a.Z1 + gj, -(cval * dz));
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    a.Z[k0 * plane + (size_t)gi0 * a.Z1 + gj0] = best.znew;
                    n_upd++;
                    int dl[kDirs];
                    Tile<real, NT> tt;
                    tt.ta = ta;
                    tt.tb = tb;
                    tt.h = h;
                    tt.wd = wd;
                    const int nd = border ? target_dirs<real, NT>(a, tt, li0, lj0, dl) : 0;
                    if (nd > 0) {
                        __threadfence();  // the window's reductions before the flags
                        atomicAdd(&a.hdr->pending, nd);
                        for (int i = 0; i < nd; i++) {
                            int dr, dc;
                            dir_offset(dl[i], dr, dc);
                            atomicAdd(a.ctl + (size_t)((ta + dr) * a.G1 + (tb + dc)) * kDirs * 32, 1);
                        }
                        n_msg += nd;
                    }
                    if (a.max_updates > 0) {
                        unsigned long long prev = atomicAdd(&a.hdr->updates_total, 1ull);
                        if ((long long)prev + 1 >= a.max_updates) set_stop(a.hdr, CSC_NOT_CONVERGED);
                    }
                    const real az = best.znew < real(0) ? -best.znew : best.znew;
                    if (a.guard_on && az > guard) set_stop(a.hdr, CSC_ERR_DIVERGED);
                }
            }
        } else {
            n_sub++;
        }
        quiet = (active || got > 0) ? 0 : quiet + 1;
        m = (m + 1 == M) ? 0 : m + 1;
        __syncthreads();
        if (quiet >= M) {
            // pause until a neighbour bumps the flag or every worker is done
            if (threadIdx.x == 0) {
                atomicSub(&a.hdr->pending, 1);
                int state = 0;
                for (;;) {
                    if (ld_relaxed(flag) != seen) {
                        atomicAdd(&a.hdr->pending, 1);
                        break;
                    }
                    if (ld_acquire(&a.hdr->pending) == 0 || ld_relaxed(&a.hdr->stop)) {
                        state = 1;
                        break;
                    }
                    if (globaltimer_ns() > deadline) {
                        set_stop(a.hdr, CSC_ERR_TIMEOUT);
                        state = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                s_ctl[2] = state;
            }
            __syncthreads();
            if (s_ctl[2]) break;
            quiet = 0;
        }
    }
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_UPDATES], (unsigned long long)n_upd);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_ITERS], (unsigned long long)n_it);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_REJECTED], (unsigned long long)n_rej);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_SUBTOL], (unsigned long long)n_sub);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_MESSAGES], (unsigned long long)n_msg);
        atomicMax(&a.hdr->wmax[0], (unsigned long long)n_it);
        atomicMax(&a.hdr->wmax[1], (unsigned long long)n_upd);
    }
}

}  // namespace csc

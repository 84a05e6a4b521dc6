// wl_walk.cuh -- the Wang-Landau walker kernel for micromagnetic lines
// (arXiv:1302.2320, the procedure around Eq. 3 and Eq. 4).
//
// One walker = one line l = S consecutive lanes of a warp ("group").  The S
// lanes evaluate the S consecutive steps t, t+1, ..., t+S-1 from the same
// state: lane m draws Philox(ctr = t+m) and computes its proposal (U[a], D[b]),
// k' and its accept decision.  The m earlier steps of the batch, if all
// rejected, each added ln f at the current bin, so lane m tests against
// ln g(k) + m ln f when k' != k (k' == k is always accepted).  The first
// accepting lane m* commits m* rejections and its accept; the next batch starts
// at t + m* + 1.  Because the random numbers are keyed by t, the committed
// chain is the sequential chain, bit for bit, for every S.  Batches never
// cross a flatness check (t multiple of C) or the end of the slice.
//
// The current bin's ln g and histogram are kept in registers (plus a pending
// count) and written back when the walker leaves the bin or reaches a check;
// every other bin is up to date in global memory.
#pragma once

#include "wl_device.cuh"

namespace wl {

template <int S>
__device__ __forceinline__ unsigned group_mask(int gbase)
{
    if constexpr (S == 32) return 0xffffffffu;
    else return ((1u << S) - 1u) << gbase;
}

// Flatness (80%/80% convention, fraction x = flat_pm/1000, exact integers):
// n visited bins, Ssum = their histogram total, c = bins with
// 1000*n*h >= flat_pm*Ssum; flat iff 1000*c >= flat_pm*n.
template <int S>
__device__ bool group_flat(const uint32_t* hist, int nbins, int m, unsigned gmask, int flat_pm)
{
    int64_t n = 0, ssum = 0;
    for (int b = m; b < nbins; b += S) {
        const uint32_t h = hist[b];
        if (h & kVisited) {
            n += 1;
            ssum += (int64_t)(h & ~kVisited);
        }
    }
    n = group_sum<S>(gmask, n);
    ssum = group_sum<S>(gmask, ssum);
    if (n == 0) return false;
    int64_t c = 0;
    const int64_t rhs = (int64_t)flat_pm * ssum;
    for (int b = m; b < nbins; b += S) {
        const uint32_t h = hist[b];
        if ((h & kVisited) && 1000 * n * (int64_t)(h & ~kVisited) >= rhs) c += 1;
    }
    c = group_sum<S>(gmask, c);
    return 1000 * c >= (int64_t)flat_pm * n;
}

// Stage step after a flat histogram: the constant shift that puts the visited
// minimum of ln g at zero stands in for the normalisation of Eq. 4 (Eq. 4 is
// applied exactly at assembly); the histogram is reset, visited bits kept.
template <int S>
__device__ void group_stage_step(int64_t* lng, uint32_t* hist, int nbins, int m, unsigned gmask)
{
    int64_t mn = INT64_MAX;
    for (int b = m; b < nbins; b += S)
        if (hist[b] & kVisited) mn = lng[b] < mn ? lng[b] : mn;
    mn = group_min<S>(gmask, mn);
    for (int b = m; b < nbins; b += S) {
        const uint32_t h = hist[b];
        if (h & kVisited) lng[b] -= mn;
        hist[b] = h & kVisited;
    }
    __syncwarp(gmask);
}

// Walk line `li` for up to A.slice_moves moves (or to its budget, or to
// convergence).  perm/sp point at the line's list and spins, in shared or
// global memory.  All lanes of the group hold identical copies of the scalar
// state.
template <int LAT, int S, bool DET, typename IDX>
__device__ void walk_line(const WalkArgs& A, int li, int m, int gbase, unsigned gmask,
                          IDX* perm, uint32_t* sp, const uint32_t* tab)
{
    const LineDesc D = A.desc[li];
    LineState* P = A.st + li;
    int64_t k = P->k, t = P->t, F = P->F, stage = P->stage, accepts = P->accepts;
    int64_t t_stage = P->t_stage, status = P->status, checks = P->checks;
    if (status != 0) return;
    const int ell = D.ell;
    const uint32_t nd = (uint32_t)(A.g.N - ell);
    int64_t* lng = A.lng + D.bin_off;
    uint32_t* hist = A.hist + D.bin_off;
    const uint2 key = make_uint2((uint32_t)ell, A.seed);
    int64_t end = t + A.slice_moves;
    if (end > A.budget) end = A.budget;

    int bc = (int)(k >> 1);
    int64_t cur = lng[bc];
    uint32_t hcur = hist[bc];
    uint32_t pend = 0;
    int stop = 0;

    while (t < end && !stop) {
        const int64_t next_check = (t / A.C + 1) * A.C;
        int64_t lim64 = next_check - t;
        if (end - t < lim64) lim64 = end - t;
        const int lim = lim64 < S ? (int)lim64 : S;

        bool acc = false, bad = false;
        uint32_t a = 0, b = 0, i = 0, j = 0;
        int kp = (int)k;
        int64_t lp = 0;
        if (m < lim) {
            const uint64_t tt = (uint64_t)(t + m);
            const uint4 r = philox4x32_10(make_uint4((uint32_t)tt, (uint32_t)(tt >> 32), 0u, 0u), key);
            a = pick(r.x, (uint32_t)ell);
            b = pick(r.y, nd);
            i = (uint32_t)perm[a];
            j = (uint32_t)perm[ell + b];
            kp = (int)k + delta_k<LAT>(A.g, sp, i, j);
            if (kp == (int)k) {
                acc = true;
            } else if ((unsigned)(kp >> 1) >= (unsigned)D.nbins) {
                bad = true;      // k' outside the line's bins: state invariant broken
            } else {
                lp = lng[kp >> 1];
                const int64_t d = lp - (cur + (int64_t)m * F);
                acc = d <= 0 || accept_uphill<DET>(d, r.z, tab, A.q, A.neg_u_log2e);
            }
        }
        if (__ballot_sync(gmask, bad)) {
            stop = 4;
            break;
        }
        unsigned bal = __ballot_sync(gmask, acc);
        if constexpr (S < 32) bal = (bal >> gbase) & ((1u << S) - 1u);
        if (bal) {
            const int ms = __ffs(bal) - 1;
            const int src = gbase + ms;
            const int kn = __shfl_sync(gmask, kp, src);
            const int64_t ln = __shfl_sync(gmask, lp, src);
            if (m == ms) {
                perm[a] = (IDX)j;
                perm[ell + b] = (IDX)i;
                sp[i >> 5] &= ~(1u << (i & 31u));
                sp[j >> 5] |= 1u << (j & 31u);
            }
            accepts += 1;
            if (kn != (int)k) {
                const uint32_t pt = pend + (uint32_t)ms;
                if (pt) {
                    if ((uint64_t)(hcur & ~kVisited) + pt >= (uint64_t)kVisited) stop = 2;
                    if (m == 0) {
                        lng[bc] = cur + (int64_t)ms * F;
                        hist[bc] = (hcur + pt) | kVisited;
                    }
                }
                k = kn;
                bc = kn >> 1;
                cur = ln + F;
                hcur = hist[bc];
                pend = 1;
            } else {
                cur += (int64_t)(ms + 1) * F;
                pend += (uint32_t)(ms + 1);
            }
            t += ms + 1;
            __syncwarp(gmask);
        } else {
            cur += (int64_t)lim * F;
            pend += (uint32_t)lim;
            t += lim;
        }
        if ((hcur & ~kVisited) + (uint64_t)pend >= (uint64_t)kVisited) stop = 2;

        if (t == next_check && !stop) {
            // flush the current bin, then test flatness over the line
            if (pend) {
                hcur = (hcur + pend) | kVisited;
                if (m == 0) {
                    lng[bc] = cur;
                    hist[bc] = hcur;
                }
                pend = 0;
            }
            __syncwarp(gmask);
            checks += 1;
            if (group_flat<S>(hist, D.nbins, m, gmask, A.flat_pm)) {
                group_stage_step<S>(lng, hist, D.nbins, m, gmask);
                F >>= 2;                     // ln f -> ln f / 4
                stage += 1;
                t_stage = t;
                cur = lng[bc];
                hcur = hist[bc];
                if (F == 0) {                // ln f < ln f_min
                    status = 1;
                    break;
                }
            }
            // stop requests are read by one lane and broadcast, so the group
            // stays converged
            int req = 0;
            if (m == 0) {
                if (A.deadline_ns && *A.deadline_ns && globaltimer_ns() > *A.deadline_ns) req = 1;
                if (A.abort_flag && *A.abort_flag) req = 3;
            }
            req = __shfl_sync(gmask, req, gbase);
            if (req) stop = req;
        }
    }
    if (pend) {
        hcur = (hcur + pend) | kVisited;
        if (m == 0) {
            lng[bc] = cur;
            hist[bc] = hcur;
        }
    }
    if (stop == 2) status = 2;
    if (stop == 4) status = 3;
    if (m == 0) {
        P->k = k;
        P->t = t;
        P->F = F;
        P->stage = stage;
        P->accepts = accepts;
        P->t_stage = t_stage;
        P->status = status;
        P->checks = checks;
        if (stop == 1) atomicOr(A.flags, 1);
        if (stop == 3) atomicOr(A.flags, 2);
        if (stop == 2) atomicOr(A.flags, 4);
        if (stop == 4) atomicOr(A.flags, 8);
    }
    __syncwarp(gmask);
}

// Copy n 32-bit words with the group's lanes (16-byte chunks when aligned).
template <int S>
__device__ __forceinline__ void group_copy(uint32_t* dst, const uint32_t* src, int nwords, int m)
{
    if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15u) == 0) {
        const int n4 = nwords >> 2;
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        for (int x = m; x < n4; x += S) d4[x] = s4[x];
        for (int x = (n4 << 2) + m; x < nwords; x += S) dst[x] = src[x];
    } else {
        for (int x = m; x < nwords; x += S) dst[x] = src[x];
    }
}

// Persistent walker: every group pops lines from the work queue until it is
// empty.  With one group and a one-entry queue the same kernel is the plain
// one-launch-per-line form.
template <int LAT, int S, bool DET, typename IDX>
__global__ void walk_kernel(const WalkArgs A)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t* tab = reinterpret_cast<uint32_t*>(smem);
    for (int x = threadIdx.x; x < kTableN; x += blockDim.x) tab[x] = A.table[x];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int m = lane % S;
    const int gbase = lane - m;
    const unsigned gmask = group_mask<S>(gbase);
    const int gid = threadIdx.x / S;
    uint8_t* slot = smem + kTableBytes + (size_t)gid * (size_t)A.slot_bytes;
    // per-line strides are padded to 16 bytes: pstride list entries, W spin words
    const int pstride = A.pstride, W = A.g.W;
    const int perm_words = (int)((size_t)pstride * sizeof(IDX) / 4);

    for (;;) {
        int qi = 0;
        if (m == 0) qi = atomicAdd(A.qnext, 1);
        qi = __shfl_sync(gmask, qi, gbase);
        if (qi >= A.nqueue) break;
        const int li = A.order[qi];
        if (A.st[li].status != 0) continue;
        IDX* gperm = reinterpret_cast<IDX*>(A.perm) + (size_t)li * pstride;
        uint32_t* gsp = A.spins + (size_t)li * W;
        if (A.stage_smem) {
            IDX* sperm = reinterpret_cast<IDX*>(slot);
            uint32_t* ssp = reinterpret_cast<uint32_t*>(slot + (size_t)perm_words * 4);
            group_copy<S>(reinterpret_cast<uint32_t*>(sperm), reinterpret_cast<const uint32_t*>(gperm),
                          perm_words, m);
            group_copy<S>(ssp, gsp, W, m);
            __syncwarp(gmask);
            walk_line<LAT, S, DET, IDX>(A, li, m, gbase, gmask, sperm, ssp, tab);
            group_copy<S>(reinterpret_cast<uint32_t*>(gperm), reinterpret_cast<const uint32_t*>(sperm),
                          perm_words, m);
            group_copy<S>(gsp, ssp, W, m);
            __syncwarp(gmask);
        } else {
            walk_line<LAT, S, DET, IDX>(A, li, m, gbase, gmask, gperm, gsp, tab);
        }
    }
}

}  // namespace wl

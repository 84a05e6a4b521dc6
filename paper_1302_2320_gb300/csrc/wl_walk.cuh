// wl_walk.cuh -- the Wang-Landau walker kernel for micromagnetic lines
// (arXiv:1302.2320, the procedure around Eq. 3 and Eq. 4).
//
// One walker = one line l = S consecutive lanes of a warp ("group").  A batch
// covers the steps t .. t+S-1:
//   parallel phase -- lane m draws Philox(ctr = t+m) and evaluates its
//     exchange proposal against the state at the start of the batch: list
//     slots a, b, sites i = U[a], j = D[b], their neighbours and the change of
//     k (all of this is independent of the acceptance decisions);
//   resolution -- the group resolves the steps in order with Eq. 3 against
//     the current k and ln g (every lane holds the same walker state), either
//     one step at a time, or in rounds: while the walker stays in its bin,
//     step m sees the ln g of step e0 plus F for each step in between, so all
//     lanes test their own step at once, a ballot finds the first accepted
//     step, the rejections before it are committed together, and the lanes
//     are re-tested only when an accepted step changes the bin.  Each walker
//     takes rounds while fewer than half of its recent steps were accepted.
//     An accepted exchange of (i_s, j_s) leaves a later proposal exact unless
//     it reuses list slot a_s or b_s or has i_s or j_s among its sites'
//     neighbours; such proposals are marked, and the batch ends at the first
//     marked one (or when a proposal's bin leaves the ln g window).
// The accepted exchanges of a batch are mutually independent and are applied
// together after the resolution.  Random numbers are keyed by t, so the committed
// chain is the sequential chain, bit for bit, for every S.  Batches never cross
// a flatness check (t multiple of C) or the end of the slice.
//
// The current bin's ln g and histogram are kept in registers (plus a pending
// count); the bins around it live in a shared-memory window that is written
// back when the walker re-centres it, at every check and at the end.
#pragma once

#include "wl_device.cuh"

namespace wl {

template <int S>
__device__ __forceinline__ unsigned group_mask(int gbase)
{
    if constexpr (S == 32) return 0xffffffffu;
    else return ((1u << S) - 1u) << gbase;
}

// The predicate of each lane of the group as bits 0 .. S-1.
template <int S>
__device__ __forceinline__ unsigned group_ballot(unsigned gmask, int gbase, bool p)
{
    const unsigned b = __ballot_sync(gmask, p);
    if constexpr (S == 32) return b;
    else return (b >> gbase) & ((1u << S) - 1u);
}

// Flatness (80%/80% convention, fraction x = flat_pm/1000, exact integers):
// n visited bins, Ssum = their histogram total, c = bins with
// 1000*n*h >= flat_pm*Ssum; flat iff 1000*c >= flat_pm*n.
template <int S>
__device__ bool group_flat(const hist_t* hist, int nbins, int m, unsigned gmask, int flat_pm)
{
    int64_t n = 0;
    uint64_t ssum = 0;
    for (int b = m; b < nbins; b += S) {
        const hist_t h = hist[b];
        if (h & kVisited) {
            n += 1;
            ssum += h & ~kVisited;
        }
    }
    n = group_sum<S>(gmask, n);
    ssum = group_sum<S>(gmask, ssum);
    if (n == 0) return false;
    int64_t c = 0;
    // products of up to ~2^77: compared in 128-bit integers
    const unsigned __int128 rhs = (unsigned __int128)flat_pm * ssum;
    const unsigned __int128 scale = (unsigned __int128)(1000 * n);
    for (int b = m; b < nbins; b += S) {
        const hist_t h = hist[b];
        if ((h & kVisited) && scale * (h & ~kVisited) >= rhs) c += 1;
    }
    c = group_sum<S>(gmask, c);
    return 1000 * c >= (int64_t)flat_pm * n;
}

// Stage step after a flat histogram: the constant shift that puts the visited
// minimum of ln g at zero stands in for the normalisation of Eq. 4 (Eq. 4 is
// applied exactly at assembly); the histogram is reset, visited bits kept.
template <int S>
__device__ void group_stage_step(int64_t* lng, hist_t* hist, int nbins, int m, unsigned gmask)
{
    int64_t mn = INT64_MAX;
    for (int b = m; b < nbins; b += S)
        if (hist[b] & kVisited) mn = lng[b] < mn ? lng[b] : mn;
    mn = group_min<S>(gmask, mn);
    for (int b = m; b < nbins; b += S) {
        const hist_t h = hist[b];
        if (h & kVisited) lng[b] -= mn;
        hist[b] = h & kVisited;
    }
    __syncwarp(gmask);
}

// Window of ln g / histogram bins a walker keeps in shared memory.  Every
// proposal lies within z bins of the current bin (|dk| <= 2z), so the window
// [wb, wb + kWin) is re-centred whenever the current bin comes within z bins of
// an edge that is not the line's own edge.

template <int S>
__device__ __forceinline__ void window_store(int64_t* wl, hist_t* wh, int64_t* lng, hist_t* hist,
                                             int wb, int wn, int m)
{
    for (int x = m; x < wn; x += S) {
        lng[wb + x] = wl[x];
        hist[wb + x] = wh[x];
    }
}

template <int S>
__device__ __forceinline__ void window_load(int64_t* wl, hist_t* wh, const int64_t* lng,
                                            const hist_t* hist, int wb, int wn, int m)
{
    for (int x = m; x < wn; x += S) {
        wl[x] = lng[wb + x];
        wh[x] = hist[wb + x];
    }
}

__device__ __forceinline__ int window_base(int bc, int nbins)
{
    int wb = bc - kWin / 2;
    if (wb > nbins - kWin) wb = nbins - kWin;
    return wb < 0 ? 0 : wb;
}

__device__ __forceinline__ uint4 philox_step(uint64_t t, uint2 key)
{
    return philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 0u, 0u), key);
}

// Walk line `li` for up to A.slice_moves moves (or to its budget, or to
// convergence).  perm/sp point at the line's list and spins (shared or global
// memory); win is the group's window (kWin int64 ln g, then kWin u64 hist).
// All lanes of the group hold identical copies of the scalar state.  The
// current bin's ln g, histogram word and pending count live in registers and
// are authoritative; every other bin is up to date in the window (inside it)
// or in global memory (outside it).
//
// Random numbers are double-buffered: lane m holds Philox(t + m) in (r0x, r0y,
// r0z) and Philox(t + S + m) in (r1x, r1y, r1z).  After a batch commits c
// steps the buffers are shifted by c with two shuffles, and the lanes whose
// entry falls past the buffered range draw Philox(t + c + S + m) -- a value
// the next batch does not use, so its latency overlaps the next batch's work.
template <int LAT, int S, bool DET, typename IDX>
__device__ void walk_line(const WalkArgs& A, int li, int m, int gbase, unsigned gmask,
                          IDX* perm, uint32_t* sp, const uint32_t* tab, uint8_t* win)
{
    constexpr int zb = Coord<LAT>::zbin;  // largest bin step of one move
    constexpr int ks = Coord<LAT>::kshift;
    const LineDesc D = A.desc[li];
    LineState* P = A.st + li;
    int64_t k = P->k, t = P->t, F = P->F, stage = P->stage, accepts = P->accepts;
    int64_t t_stage = P->t_stage, status = P->status, checks = P->checks;
    int64_t batches = P->batches;
    if (status != 0) return;
    const int ell = D.ell, nbins = D.nbins;
    const uint32_t nd = (uint32_t)(A.g.N - ell);
    int64_t* lng = A.lng + D.bin_off;
    hist_t* hist = A.hist + D.bin_off;
    int64_t* wl = reinterpret_cast<int64_t*>(win);
    hist_t* wh = reinterpret_cast<hist_t*>(win + kWin * 8);
    const uint2 key = make_uint2((uint32_t)ell, A.seed);
    int64_t end = t + A.slice_moves;
    if (end > A.budget) end = A.budget;

    int bc = (int)(k >> ks);
    int wb = window_base(bc, nbins);
    const int wn = nbins < kWin ? nbins : kWin;
    window_load<S>(wl, wh, lng, hist, wb, wn, m);
    __syncwarp(gmask);
    int64_t cur = wl[bc - wb];
    hist_t hcur = wh[bc - wb];
    uint32_t pend = 0;
    int stop = 0;
    bool by_rounds = false;               // resolution chosen from the acceptance rate
    int rate_acc = 0, rate_steps = 0;

    uint4 r0 = philox_step((uint64_t)(t + m), key);
    uint4 r1 = make_uint4(0u, 0u, 0u, 0u);
    uint64_t tf = (uint64_t)(t + S + m);   // pending draw for r1
    bool needf = true;

    while (t < end && !stop) {
        const int64_t next_check = (t / A.C + 1) * A.C;
        const int64_t seg_end = next_check < end ? next_check : end;
        int left = (int)(seg_end - t);    // moves before the next check or the slice end

        while (left > 0) {
            const int lim = left < S ? left : S;
            // the pending draw (independent of this batch)
            const uint4 rf = philox_step(tf, key);
            // -- parallel phase: lane m proposes step t + m against the state at
            //    the start of the batch (list slots a, b, sites i, j, their
            //    neighbours and the change of k)
            const uint32_t a = pick(r0.x, (uint32_t)ell);
            const uint32_t b = pick(r0.y, nd);
            const uint32_t i = (uint32_t)perm[a];
            const uint32_t j = (uint32_t)perm[ell + b];
            constexpr int zc = Coord<LAT>::z;
            uint32_t ni[zc], nj[zc];
            const int dk = delta_k_nb<LAT>(A.g, sp, i, j, ni, nj);
            if (needf) r1 = rf;
            // -- resolution: the steps in order with Eq. 3 against the current k
            //    and ln g (every lane holds the same walker state).  An accepted
            //    exchange of (i_s, j_s) leaves a later proposal exact unless it
            //    reuses list slot a_s or b_s or one of i_s, j_s neighbours its
            //    sites; such proposals are marked, and the batch ends at the
            //    first marked one.  Two equivalent ways, chosen per walker:
            unsigned inv = 0u, accm = 0u;
            int c = lim;
            if (A.resolve == 2 || (A.resolve == 0 && by_rounds)) {
                // Rounds.  While the walker keeps its bin, step m sees the state
                // of step e0 with F added once per step in between (a rejection
                // or an accepted exchange with dk = 0 both visit the current
                // bin), so every lane tests its own step at once.  The first lane
                // that accepts, leaves the window or was marked ends the round,
                // and the rejections before it are committed together.  Lanes
                // are tested again only after an accepted step changes the bin.
                const unsigned live = lim >= 32 ? 0xffffffffu : ((1u << lim) - 1u);
                unsigned evb = 0u;
                int pk = 0;                // (dk + 64) << 2 | kind of this lane's step
                long long lpm = 0;         // ln g of its target bin
                int e0 = 0;
                bool eval = true;
                for (int round = 0; ; ++round) {
                    if (round > S) {       // cannot happen: e0 grows every round
                        stop = 4;
                        c = e0;
                        break;
                    }
                    if (eval) {
                        // kind: 0 accepted, 1 off the window, 2 outside the line,
                        // -1 rejected; without branches (a bin outside the window
                        // reads the current bin's slot, always inside, and is
                        // not used; dk = 0 is accepted)
                        const int bp = ((int)k + dk) >> ks;
                        const int wx = bp - wb;
                        const bool brk = (unsigned)bp >= (unsigned)nbins;
                        const bool off = (unsigned)wx >= (unsigned)wn;
                        lpm = wl[(brk || off) ? bc - wb : wx];
                        const int64_t d = lpm - (cur + (int64_t)(m - e0) * F);
                        const bool up = accept_uphill<DET>(d, r0.z, tab, A.q, A.neg_u_log2e);
                        const int kind = dk == 0 ? 0 : brk ? 2 : off ? 1 : (d <= 0 || up) ? 0 : -1;
                        pk = ((dk + 64) << 2) | (kind & 3);
                        evb = group_ballot<S>(gmask, gbase, kind >= 0);
                        eval = false;
                    }
                    const unsigned ev = (evb | inv) & live & ~((1u << e0) - 1u);
                    if (ev == 0u) {        // the rest of the batch is rejected
                        cur += (int64_t)(lim - e0) * F;
                        pend += (uint32_t)(lim - e0);
                        break;
                    }
                    const int e = __ffs(ev) - 1;
                    cur += (int64_t)(e - e0) * F;      // rejections e0 .. e-1
                    pend += (uint32_t)(e - e0);
                    const unsigned bit = 1u << e;
                    if (inv & bit) {
                        c = e;
                        break;
                    }
                    const int src = gbase + e;
                    const int code = __shfl_sync(gmask, pk, src);
                    const int64_t lpe = __shfl_sync(gmask, lpm, src);
                    if ((code & 3) == 2) {             // invariant broken
                        stop = 4;
                        c = e;
                        break;
                    }
                    if ((code & 3) == 1) {             // walked off the window
                        c = e;
                        break;
                    }
                    accm |= bit;
                    const int dke = (code >> 2) - 64;
                    if (dke != 0) {
                        // leave the current bin: its ln g and histogram go to the window
                        const int kp = (int)k + dke;
                        if ((hcur & ~kVisited) + pend >= kVisited) stop = 2;
                        if (pend) hcur = (hcur + pend) | kVisited;
                        wl[bc - wb] = cur;
                        wh[bc - wb] = hcur;
                        k = kp;
                        bc = kp >> ks;
                        cur = lpe + F;
                        hcur = wh[bc - wb];
                        pend = 1u;
                        eval = true;
                    } else {
                        cur += F;
                        pend += 1u;
                    }
                    // later proposals that the accepted exchange of (i_e, j_e) affects
                    const uint32_t as = __shfl_sync(gmask, a, src), bs = __shfl_sync(gmask, b, src);
                    const uint32_t is = __shfl_sync(gmask, i, src), js = __shfl_sync(gmask, j, src);
                    bool conf = (a == as) | (b == bs);
#pragma unroll
                    for (int q = 0; q < zc; ++q)
                        conf |= (ni[q] == is) | (ni[q] == js) | (nj[q] == is) | (nj[q] == js);
                    inv |= group_ballot<S>(gmask, gbase, conf && m > e);
                    e0 = e + 1;
                    if (stop) {
                        c = e0;
                        break;
                    }
                    if (e0 >= lim) break;
                }
            } else {
                // Steps one at a time; step s's change of k and random word are
                // shuffled one step ahead.
                int dkn = __shfl_sync(gmask, dk, gbase);
                uint32_t rzn = __shfl_sync(gmask, r0.z, gbase);
                for (int s = 0; s < lim; ++s) {
                    const int src = gbase + s;
                    const int dks = dkn;
                    const uint32_t rzs = rzn;
                    const int nxt = gbase + (s + 1 < S ? s + 1 : s);
                    dkn = __shfl_sync(gmask, dk, nxt);
                    rzn = __shfl_sync(gmask, r0.z, nxt);
                    if ((inv >> s) & 1u) {
                        c = s;
                        break;
                    }
                    const int kp = (int)k + dks;
                    bool acc = true;
                    int64_t lp = 0;
                    if (dks != 0) {
                        const int bp = kp >> ks;
                        const int wx = bp - wb;
                        if ((unsigned)bp >= (unsigned)nbins) {      // invariant broken
                            stop = 4;
                            c = s;
                            break;
                        }
                        if ((unsigned)wx >= (unsigned)wn) {        // walked off the window
                            c = s;
                            break;
                        }
                        lp = wl[wx];
                        const int64_t d = lp - cur;
                        acc = d <= 0 || accept_uphill<DET>(d, rzs, tab, A.q, A.neg_u_log2e);
                    }
                    if (!acc) {
                        cur += F;
                        pend += 1u;
                        continue;
                    }
                    accm |= 1u << s;
                    if (dks != 0) {
                        // leave the current bin: its ln g and histogram go to the window
                        if ((hcur & ~kVisited) + pend >= kVisited) stop = 2;
                        if (pend) hcur = (hcur + pend) | kVisited;
                        wl[bc - wb] = cur;
                        wh[bc - wb] = hcur;
                        k = kp;
                        bc = kp >> ks;
                        cur = lp + F;
                        hcur = wh[bc - wb];
                        pend = 1u;
                    } else {
                        cur += F;
                        pend += 1u;
                    }
                    // later proposals that the accepted exchange of (i_s, j_s) affects
                    const uint32_t as = __shfl_sync(gmask, a, src), bs = __shfl_sync(gmask, b, src);
                    const uint32_t is = __shfl_sync(gmask, i, src), js = __shfl_sync(gmask, j, src);
                    bool conf = (a == as) | (b == bs);
#pragma unroll
                    for (int q = 0; q < zc; ++q)
                        conf |= (ni[q] == is) | (ni[q] == js) | (nj[q] == is) | (nj[q] == js);
                    inv |= group_ballot<S>(gmask, gbase, conf && m > s);
                    if (stop) {
                        c = s + 1;
                        break;
                    }
                }
            }
            if (c == 0) stop = 4;                  // lane 0 is always evaluable
            // apply the accepted exchanges (mutually independent) to lists and spins
            if ((accm >> m) & 1u) {
                perm[a] = (IDX)j;
                perm[ell + b] = (IDX)i;
                atomicAnd(&sp[i >> 5], ~(1u << (i & 31u)));
                atomicOr(&sp[j >> 5], 1u << (j & 31u));
            }
            accepts += __popc(accm);
            // rounds pay per accepted step, single steps per step: pick rounds
            // while fewer than half of the recent steps were accepted
            rate_acc += __popc(accm);
            rate_steps += c;
            if (rate_steps >= 512) {
                by_rounds = 2 * rate_acc < rate_steps;
                rate_acc = rate_steps = 0;
            }
            __syncwarp(gmask);
            if ((bc - zb < wb && wb > 0) || (bc + zb >= wb + kWin && wb + kWin < nbins)) {
                // re-centre the window (the current bin stays in registers)
                window_store<S>(wl, wh, lng, hist, wb, wn, m);
                __syncwarp(gmask);
                wb = window_base(bc, nbins);
                window_load<S>(wl, wh, lng, hist, wb, wn, m);
                __syncwarp(gmask);
            }
            // shift the random-number buffers by c: lane m now needs steps
            // t + c + m (r0) and t + c + S + m (r1)
            {
                const int srcm = m + c;                       // < 2S
                const int sl = gbase + (srcm & (S - 1));
                const uint32_t ax = __shfl_sync(gmask, r0.x, sl), ay = __shfl_sync(gmask, r0.y, sl),
                               az = __shfl_sync(gmask, r0.z, sl);
                const uint32_t bx = __shfl_sync(gmask, r1.x, sl), by = __shfl_sync(gmask, r1.y, sl),
                               bz = __shfl_sync(gmask, r1.z, sl);
                needf = srcm >= S;
                r0 = needf ? make_uint4(bx, by, bz, 0u) : make_uint4(ax, ay, az, 0u);
                r1 = make_uint4(bx, by, bz, 0u);
                tf = (uint64_t)(t + c + S + m);
            }
            t += c;
            left -= c;
            batches += 1;
            if (stop) break;
        }
        if (stop) break;

        if (t == next_check) {
            // current bin -> window -> global, then test flatness over the line
            if ((hcur & ~kVisited) + pend >= kVisited) {
                stop = 2;
                break;
            }
            if (pend) hcur = (hcur + pend) | kVisited;
            pend = 0;
            if (m == 0) {
                wl[bc - wb] = cur;
                wh[bc - wb] = hcur;
            }
            __syncwarp(gmask);
            window_store<S>(wl, wh, lng, hist, wb, wn, m);
            __syncwarp(gmask);
            checks += 1;
            const bool flat = group_flat<S>(hist, nbins, m, gmask, A.flat_pm);
            if (!flat && A.same_f_resets > 0 && (t - t_stage) / A.C <= A.same_f_resets) {
                // extra reset at unchanged f within the first R checks of a
                // stage (the remark after Eq. 4): histogram reset, ln g shifted
                group_stage_step<S>(lng, hist, nbins, m, gmask);
                window_load<S>(wl, wh, lng, hist, wb, wn, m);
                __syncwarp(gmask);
                cur = wl[bc - wb];
                hcur = wh[bc - wb];
            }
            if (flat) {
                group_stage_step<S>(lng, hist, nbins, m, gmask);
                F >>= 2;                     // ln f -> ln f / 4
                stage += 1;
                t_stage = t;
                window_load<S>(wl, wh, lng, hist, wb, wn, m);
                __syncwarp(gmask);
                cur = wl[bc - wb];
                hcur = wh[bc - wb];
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
    // current bin -> window -> global
    if (stop != 4) {
        if (pend) hcur = (hcur + pend) | kVisited;
        if (m == 0) {
            wl[bc - wb] = cur;
            wh[bc - wb] = hcur;
        }
        __syncwarp(gmask);
        window_store<S>(wl, wh, lng, hist, wb, wn, m);
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
        P->batches = batches;
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
    // per-group slot: window, then (when staged) the list and the spins
    uint8_t* slot = smem + kTableBytes + (size_t)gid * (size_t)A.slot_bytes;
    uint8_t* win = slot;
    slot += kWinBytes;
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
            walk_line<LAT, S, DET, IDX>(A, li, m, gbase, gmask, sperm, ssp, tab, win);
            group_copy<S>(reinterpret_cast<uint32_t*>(gperm), reinterpret_cast<const uint32_t*>(sperm),
                          perm_words, m);
            group_copy<S>(gsp, ssp, W, m);
            __syncwarp(gmask);
        } else {
            walk_line<LAT, S, DET, IDX>(A, li, m, gbase, gmask, gperm, gsp, tab, win);
        }
    }
}

}  // namespace wl

// wl_walk.cuh -- the Wang-Landau walker kernel for micromagnetic lines
// (arXiv:1302.2320, the procedure around Eq. 3 and Eq. 4).
//
// One walker = one line l = S consecutive lanes of a warp ("group").  A batch
// covers the steps t .. t+S-1:
//   draw -- lane m holds the random numbers of step t+m, drawn one batch
//     ahead: the list slots a, b and dmax, the largest ln g increase that
//     Eq. 3 accepts with this step's random word (see dmax_det / dmax_prod);
//   propose -- lane m evaluates its exchange against the state at the start of
//     the batch: sites i = U[a], j = D[b], their neighbours and the change of
//     k;
//   resolve -- while the walker stays in its bin, step m sees that bin's ln g
//     plus F for every step in between (a rejection and an accepted exchange
//     with the same k both visit the current bin), so every lane tests its own
//     step at once (ln g(target) <= ln g(current) + dmax); a ballot finds the
//     first accepted step, the rejections before it are committed together,
//     and the lanes are tested again only when an accepted step changes the
//     bin or the proposals.
// An accepted exchange of (i_e, j_e) changes a later proposal in two ways.  If
// the proposal reuses list slot a_e or b_e (equivalently: names site i_e or
// j_e, the lists holding distinct sites) its sites are no longer U[a], D[b]:
// the batch is cut short before it.  If one of i_e, j_e neighbours its sites,
// its change of k is off by 2 for every such neighbour (i_e turned down, j_e
// up): the later lanes correct it in place and are tested again.  The later
// proposals an exchange may affect are found with 2z equality tests per lane,
// or (TBL, the tail shape: one walker per block) with two loads from a
// shared-memory table that lists, per site, the lanes having it among their
// sites or their neighbours.  The exchanges accepted in a batch touch distinct
// slots and distinct sites, so they are applied together after the resolution.
// Random numbers are keyed by t, so the committed chain is the sequential
// chain, bit for bit, for every S and both forms.  Batches never cross a
// flatness check (t multiple of C) or the end of the slice.
//
// The current bin's ln g and its visits not yet counted live in registers; the
// bins around it live in a shared-memory window (ln g, and the histogram counts
// added since the window was loaded: the visits to a bin the walker left are
// added by the lane of the step that left it, at the end of the batch), written
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
// an edge that is not the line's own edge.  The window holds ln g and the
// counts added since it was loaded; storing it adds the counts to the global
// histogram (a bin with a count is marked visited) and zeroes them.  Counts
// reaching 2^62 (far beyond any run) are reported as an overflow.
template <int S>
__device__ __forceinline__ bool window_store(int64_t* wl, uint32_t* wd, int64_t* lng, hist_t* hist,
                                             int wb, int wn, int m)
{
    bool ovf = false;
    for (int x = m; x < wn; x += S) {
        lng[wb + x] = wl[x];
        const uint32_t add = wd[x];
        if (add) {
            const hist_t h = hist[wb + x] + add;
            ovf |= (h & ~kVisited) >= (1ull << 62);
            hist[wb + x] = h | kVisited;
            wd[x] = 0u;
        }
    }
    return ovf;
}

template <int S>
__device__ __forceinline__ void window_load(int64_t* wl, uint32_t* wd, const int64_t* lng, int wb,
                                            int wn, int m)
{
    for (int x = m; x < wn; x += S) {
        wl[x] = lng[wb + x];
        wd[x] = 0u;
    }
}

__device__ __forceinline__ int window_base(int bc, int nbins)
{
    int wb = bc - kWin / 2;
    if (wb > nbins - kWin) wb = nbins - kWin;
    return wb < 0 ? 0 : wb;
}

template <bool DET>
__device__ __forceinline__ Draw draw_step(uint64_t t, uint2 key, uint32_t ell, uint32_t nd,
                                          const WalkArgs& A)
{
    const uint4 r = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 0u, 0u), key);
    Draw d;
    d.a = pick(r.x, ell);
    d.b = pick(r.y, nd);
    d.dmax = DET ? dmax_det(r.z, A.table, A.q, A.seg_per_log2) : dmax_prod(r.z, A.inv_u);
    return d;
}

template <int S>
__device__ __forceinline__ Draw shfl_draw(unsigned gmask, const Draw& d, int src)
{
    Draw o;
    o.a = __shfl_sync(gmask, d.a, src);
    o.b = __shfl_sync(gmask, d.b, src);
    o.dmax = __shfl_sync(gmask, d.dmax, src);
    return o;
}

// Walk line `li` for up to A.slice_moves moves (or to its budget, or to
// convergence).  perm/sp point at the line's list and spins (shared or global
// memory); win is the group's window (kWin int64 ln g, then kWin u32 counts).
// All lanes of the group hold identical copies of the scalar state.
//
// Draws are double-buffered: lane m holds the draw of step t + m in d0 and of
// t + S + m in d1.  After a batch commits c steps the buffers shift by c (a
// plain copy when c = S, the usual case), and the lanes whose entry falls past
// the buffered range take the draw of step t + c + S + m, computed at the
// start of the next batch so its latency overlaps that batch's work.
template <int LAT, int S, bool DET, typename IDX, bool TBL>
__device__ void walk_line(const WalkArgs& A, int li, int m, int gbase, unsigned gmask,
                          IDX* perm, uint32_t* sp, uint8_t* win, uint32_t* tbl)
{
    constexpr int zb = Coord<LAT>::zbin;  // largest bin step of one move
    constexpr int ks = Coord<LAT>::kshift;
    constexpr int zc = Coord<LAT>::z;
    constexpr bool kPack = sizeof(IDX) == 2;   // slots and sites fit 16 bits
    const LineDesc D = A.desc[li];
    LineState* P = A.st + li;
    int64_t t = P->t, F = P->F, stage = P->stage, accepts = P->accepts;
    int64_t t_stage = P->t_stage, status = P->status, checks = P->checks;
    int64_t batches = P->batches;
    int k = (int)P->k;
    if (status != 0) return;
    const int ell = D.ell, nbins = D.nbins;
    const uint32_t nd = (uint32_t)(A.g.N - ell);
    int64_t* lng = A.lng + D.bin_off;
    hist_t* hist = A.hist + D.bin_off;
    int64_t* wl = reinterpret_cast<int64_t*>(win);
    uint32_t* wd = reinterpret_cast<uint32_t*>(win + kWin * 8);
    const uint2 key = make_uint2((uint32_t)ell, A.seed);
    int64_t end = t + A.slice_moves;
    if (end > A.budget) end = A.budget;
    // flatness check interval of this line: longer for lines with more bins
    const int64_t C = A.C_per_bin > 0 && A.C_per_bin * nbins > A.C ? A.C_per_bin * nbins : A.C;

    int bc = k >> ks;
    int wb = window_base(bc, nbins);
    const int wn = nbins < kWin ? nbins : kWin;
    window_load<S>(wl, wd, lng, wb, wn, m);
    __syncwarp(gmask);
    int64_t cur = wl[bc - wb];    // ln g of the current bin, every visit included
    int pend = 0;                 // visits to the current bin not yet in the window
    int stop = 0;
    int64_t mF = (int64_t)m * F;

    Draw d0 = draw_step<DET>((uint64_t)(t + m), key, (uint32_t)ell, nd, A);
    Draw d1{};
    uint64_t tf = (uint64_t)(t + S + m);   // pending draw for d1
    bool needf = true;

    while (t < end && !stop) {
        const int64_t next_check = (t / C + 1) * C;
        const int64_t seg_end = next_check < end ? next_check : end;
        int left = (int)(seg_end - t);    // moves before the next check or the slice end

        while (left > 0) {
            const int lim = left < S ? left : S;
            // the pending draw (independent of this batch)
            const Draw df = draw_step<DET>(tf, key, (uint32_t)ell, nd, A);
            // -- propose: step t + m against the state at the start of the batch
            const uint32_t a = d0.a, b = d0.b;
            const uint32_t i = (uint32_t)perm[a];
            const uint32_t j = (uint32_t)perm[ell + b];
            uint32_t ni[zc], nj[zc];
            int dk = delta_k_nb<LAT>(A.g, sp, i, j, ni, nj);
            if (needf) d1 = df;
            // accepted iff ln g(target) <= ln g(current before step m) + dmax, and
            // ln g(current before step m) = u + m F while the walker keeps its bin
            const int64_t base = mF + d0.dmax;
            // U and D are lists of distinct sites, so a later proposal reuses
            // list slot a_e (b_e) of an accepted exchange iff its i (j) is i_e (j_e)
            const uint32_t ij = kPack ? (i | (j << 16)) : i;
            if constexpr (TBL) {
                // conflict filter: for every site, the lanes that have it among
                // their sites or their sites' neighbours (hashed by the low bits);
                // an accepted exchange looks up its own two sites
                const uint32_t tm = (uint32_t)A.tbl_mask, bit = 1u << m;
#pragma unroll
                for (int q = 0; q < zc; ++q) {
                    atomicOr(&tbl[ni[q] & tm], bit);
                    atomicOr(&tbl[nj[q] & tm], bit);
                }
                atomicOr(&tbl[i & tm], bit);
                atomicOr(&tbl[j & tm], bit);
                __syncwarp(gmask);
            }
            int rec_x = 0;        // the bin this lane's step left, and its visits (counted at the end)
            uint32_t rec_c = 0u;
            // -- resolve.  One pass of the loop handles one accepted step (an
            // event): the walker's state is updated by selects, the later lanes
            // are evaluated again for the next event, and only the rare cases
            // (off the window, a conflicting later proposal) branch.  Every
            // branch depends on ballots or on values all lanes hold alike.
            int lim_eff = lim;                                   // cut short by a reused slot
            unsigned live = lim >= 32 ? 0xffffffffu : ((1u << lim) - 1u);
            unsigned done = 0u;                                  // steps resolved so far
            int64_t u = cur;      // ln g of the current bin before step 0, shifted as above
            int ent = -pend;      // batch step at which the walker entered its bin
            int kw = k - (wb << ks);                             // k relative to the window
            unsigned accm = 0u;
            int c = 0;
            int64_t v;            // ln g of the target bin - m F
            unsigned evb, offb;
            {
                const int wx = (kw + dk) >> ks;
                const bool off = (unsigned)wx >= (unsigned)wn;
                const int64_t ld = wl[off ? (kw >> ks) : wx];
                v = ld - mF;
                evb = group_ballot<S>(gmask, gbase, (dk == 0) | off | (ld <= u + base));
                offb = group_ballot<S>(gmask, gbase, off);
            }
            for (;;) {
                const unsigned ev = evb & live & ~done;
                if (ev == 0u) {                      // the rest of the batch is rejected
                    c = lim_eff;
                    break;
                }
                const int e = __ffs(ev) - 1;
                const int src = gbase + e;
                const int dke = __shfl_sync(gmask, dk, src);
                const int64_t ve = __shfl_sync(gmask, v, src);
                const uint32_t ije = __shfl_sync(gmask, ij, src);
                uint32_t je = 0;
                if constexpr (!kPack) je = __shfl_sync(gmask, j, src);
                const bool offe = (offb >> e) & 1u;  // walked off the window: ends the batch at e
                // accepted step e: a new bin means steps e0 .. e-1 were rejections in the old one
                const bool mv = (dke != 0) & !offe;
                const int x = kw >> ks;
                if (mv) wl[x] = u + (int64_t)e * F;
                if (mv & (m == e)) {
                    rec_x = x;
                    rec_c = (uint32_t)(e - ent);
                }
                const int dkm = mv ? dke : 0;
                k += dkm;
                kw += dkm;
                u = mv ? ve : u;
                ent = mv ? e : ent;
                accm |= 1u << e;                     // withdrawn below if e walked off the window
                done = (2u << e) - 1u;
                // the later lanes against the new state
                int wx = (kw + dk) >> ks;
                bool off = (unsigned)wx >= (unsigned)wn;
                int64_t ld = wl[off ? (kw >> ks) : wx];
                bool acc = (dk == 0) | off | (ld <= u + base);
                // later proposals: one that reuses a slot of the exchange cuts the
                // batch short before it, one next to it gets its change of k shifted
                const uint32_t ie = kPack ? (ije & 0xFFFFu) : ije;
                if constexpr (kPack) je = ije >> 16;
                const uint32_t xs = ij ^ ije;
                bool conflict;
                if constexpr (TBL) {
                    // lanes that may be affected (a superset); tested exactly below
                    const uint32_t tm = (uint32_t)A.tbl_mask;
                    conflict = ((tbl[ie & tm] | tbl[je & tm]) & live & ~done) != 0u;
                }
                bool n0 = false, n1 = false, n2 = false, n3 = false, slot = false;
                if constexpr (!TBL) {
                    slot = kPack ? (((xs & 0xFFFFu) == 0u) | ((xs >> 16) == 0u)) : ((xs == 0u) | (j == je));
#pragma unroll
                    for (int q = 0; q < zc; ++q) {
                        n0 |= ni[q] == ie;
                        n1 |= ni[q] == je;
                        n2 |= nj[q] == ie;
                        n3 |= nj[q] == je;
                    }
                }
                if (offe) {
                    if ((unsigned)((k + dke) >> ks) >= (unsigned)nbins) stop = 4;   // invariant broken
                    accm &= ~(1u << e);
                    c = e;
                    break;
                }
                if constexpr (!TBL)
                    conflict = (group_ballot<S>(gmask, gbase, slot | (n0 | n1) | (n2 | n3)) & live & ~done) != 0u;
                if (conflict) {
                    if constexpr (TBL)
                        slot = kPack ? (((xs & 0xFFFFu) == 0u) | ((xs >> 16) == 0u)) : ((xs == 0u) | (j == je));
                    const unsigned sm = group_ballot<S>(gmask, gbase, slot) & live & ~done;
                    if (sm) {
                        lim_eff = __ffs(sm) - 1;             // > e
                        live = (1u << lim_eff) - 1u;
                    }
                    int cor = 0;
#pragma unroll
                    for (int q = 0; q < zc; ++q)
                        cor += (int)(nj[q] == ie) - (int)(ni[q] == ie) + (int)(ni[q] == je) -
                               (int)(nj[q] == je);
                    dk += 2 * cor;
                    wx = (kw + dk) >> ks;
                    off = (unsigned)wx >= (unsigned)wn;
                    ld = wl[off ? (kw >> ks) : wx];
                    acc = (dk == 0) | off | (ld <= u + base);
                }
                v = ld - mF;
                evb = group_ballot<S>(gmask, gbase, acc);
                offb = group_ballot<S>(gmask, gbase, off);
                // no step left: the next pass finds no event and ends the batch
            }
            bc = k >> ks;
            cur = u + (int64_t)c * F;
            pend = c - ent;
            if (c == 0) stop = 4;                  // step t always fits the window
            // visits to the bins the walker left in this batch, one lane per bin left
            __syncwarp(gmask);
            if (rec_c) atomicAdd(wd + rec_x, rec_c);
            if constexpr (TBL) {
                const uint32_t tm = (uint32_t)A.tbl_mask;
#pragma unroll
                for (int q = 0; q < zc; ++q) {
                    tbl[ni[q] & tm] = 0u;
                    tbl[nj[q] & tm] = 0u;
                }
                tbl[i & tm] = 0u;
                tbl[j & tm] = 0u;
            }
            // apply the accepted exchanges (distinct slots, distinct sites)
            if ((accm >> m) & 1u) {
                perm[a] = (IDX)j;
                perm[ell + b] = (IDX)i;
                atomicAnd(&sp[i >> 5], ~(1u << (i & 31u)));
                atomicOr(&sp[j >> 5], 1u << (j & 31u));
            }
            accepts += __popc(accm);
            __syncwarp(gmask);
            if ((bc - zb < wb && wb > 0) || (bc + zb >= wb + kWin && wb + kWin < nbins)) {
                // re-centre the window (the current bin stays in registers)
                if (group_ballot<S>(gmask, gbase, window_store<S>(wl, wd, lng, hist, wb, wn, m))) stop = 2;
                __syncwarp(gmask);
                wb = window_base(bc, nbins);
                window_load<S>(wl, wd, lng, wb, wn, m);
                __syncwarp(gmask);
            }
            // shift the draw buffers by c: lane m now needs steps t + c + m (d0)
            // and t + c + S + m (d1)
            if (c == S) {
                d0 = d1;
                needf = true;
            } else {
                const int srcm = m + c;                       // < 2S
                const int sl = gbase + (srcm & (S - 1));
                const Draw x0 = shfl_draw<S>(gmask, d0, sl);
                const Draw x1 = shfl_draw<S>(gmask, d1, sl);
                needf = srcm >= S;
                d0 = needf ? x1 : x0;
                d1 = x1;
            }
            tf = (uint64_t)(t + c + S + m);
            t += c;
            left -= c;
            batches += 1;
            if (stop) break;
        }
        if (stop) break;

        if (t == next_check) {
            // current bin -> window -> global, then test flatness over the line
            __syncwarp(gmask);
            if (m == 0) {
                wl[bc - wb] = cur;
                wd[bc - wb] += (uint32_t)pend;
            }
            pend = 0;
            __syncwarp(gmask);
            if (group_ballot<S>(gmask, gbase, window_store<S>(wl, wd, lng, hist, wb, wn, m))) {
                stop = 2;
                break;
            }
            __syncwarp(gmask);
            checks += 1;
            const bool flat = group_flat<S>(hist, nbins, m, gmask, A.flat_pm);
            if (!flat && A.same_f_resets > 0 && (t - t_stage) / C <= A.same_f_resets) {
                // extra reset at unchanged f within the first R checks of a
                // stage (the remark after Eq. 4): histogram reset, ln g shifted
                group_stage_step<S>(lng, hist, nbins, m, gmask);
                window_load<S>(wl, wd, lng, wb, wn, m);
                __syncwarp(gmask);
                cur = wl[bc - wb];
            }
            if (flat) {
                group_stage_step<S>(lng, hist, nbins, m, gmask);
                F >>= 2;                     // ln f -> ln f / 4
                mF = (int64_t)m * F;
                stage += 1;
                t_stage = t;
                window_load<S>(wl, wd, lng, wb, wn, m);
                __syncwarp(gmask);
                cur = wl[bc - wb];
                if (F == 0) {                // ln f < ln f_min
                    status = 1;
                    break;
                }
            }
            // stop requests are read by one lane and broadcast, so the group
            // stays converged; a time-limited slice ends here without an error
            int req = 0;
            if (m == 0) {
                const uint64_t now = globaltimer_ns();
                if (A.slice_end_ns && *A.slice_end_ns && now > *A.slice_end_ns) req = 5;
                if (A.deadline_ns && *A.deadline_ns && now > *A.deadline_ns) req = 1;
                if (A.abort_flag && *A.abort_flag) req = 3;
            }
            req = __shfl_sync(gmask, req, gbase);
            if (req) stop = req;
        }
    }
    // current bin -> window -> global
    if (stop != 4) {
        __syncwarp(gmask);
        if (m == 0) {
            wl[bc - wb] = cur;
            wd[bc - wb] += (uint32_t)pend;
        }
        __syncwarp(gmask);
        if (group_ballot<S>(gmask, gbase, window_store<S>(wl, wd, lng, hist, wb, wn, m)) && stop == 0)
            stop = 2;
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
template <int LAT, int S, bool DET, typename IDX, bool TBL>
__global__ void walk_kernel(const WalkArgs A)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int m = lane % S;
    const int gbase = lane - m;
    const unsigned gmask = group_mask<S>(gbase);
    const int gid = threadIdx.x / S;
    // per-group slot: window, then (when staged) the list and the spins
    uint8_t* slot = smem + (size_t)gid * (size_t)A.slot_bytes;
    uint8_t* win = slot;
    slot += kWinBytes;
    uint32_t* tbl = nullptr;
    if constexpr (TBL) {
        // the conflict filter table starts empty and is left empty by every batch
        tbl = reinterpret_cast<uint32_t*>(slot);
        const int words = A.tbl_mask + 1;
        for (int x = m; x < words; x += S) tbl[x] = 0u;
        __syncwarp(gmask);
        slot += (size_t)words * 4;
    }
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
            walk_line<LAT, S, DET, IDX, TBL>(A, li, m, gbase, gmask, sperm, ssp, win, tbl);
            group_copy<S>(reinterpret_cast<uint32_t*>(gperm), reinterpret_cast<const uint32_t*>(sperm),
                          perm_words, m);
            group_copy<S>(gsp, ssp, W, m);
            __syncwarp(gmask);
        } else {
            walk_line<LAT, S, DET, IDX, TBL>(A, li, m, gbase, gmask, gperm, gsp, win, tbl);
        }
    }
}

}  // namespace wl

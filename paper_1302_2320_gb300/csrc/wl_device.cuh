// wl_device.cuh -- device building blocks of the micromagnetic-line
// Wang-Landau walker (arXiv:1302.2320): Philox4x32-10, lattice geometry on
// bit-packed spins, the change of k under a spin exchange, the acceptance of
// Eq. 3 as a threshold on the ln g difference, and warp-group helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wl {

using hist_t = uint64_t;                       // histogram word: count, bit 63 = ever visited
constexpr hist_t kVisited = 1ull << 63;
constexpr int kTableN = 4096;
constexpr int kTableBytes = kTableN * 4;     // entries 1..4095 as u32; entry 0 is 2^32

// kSquareP2: the square lattice when L is a power of two (coordinates by
// shift and mask); the same lattice and bond set as kSquare.
// kSquareOpen: the square lattice with open boundaries (sites on an edge have
// fewer neighbours; k takes every value, so bins have step 1).
enum LatticeType : int { kSquare = 0, kTriangular = 1, kCubic = 2, kSquareP2 = 3, kSquareOpen = 4 };

// Per-walker window in shared memory: ln g (int64) of kWin bins, then the
// histogram counts (u32) the walker added to them since the window was loaded.
constexpr int kWin = 64;
constexpr int kWinBytes = kWin * 12;

// Per-line scalar state (device, one per walked line).
struct LineState {
    int64_t k;         // current number of unhappy bonds
    int64_t t;         // move attempts made (the Philox step counter)
    int64_t F;         // ln f in units of u = ln f_min
    int64_t stage;     // completed flat histograms
    int64_t accepts;   // accepted proposals
    int64_t t_stage;   // t at the start of the current stage
    int64_t status;    // 0 running, 1 converged, 2 histogram overflow, 3 invariant broken
    int64_t checks;    // flatness checks made
    int64_t batches;   // speculative batches evaluated (diagnostic)
};

struct LineDesc {
    int64_t bin_off;   // first bin of this line in the ragged lng/hist arrays
    int32_t ell;       // number of up spins
    int32_t nbins;     // bins k = 0, 2, ..., 2*(nbins-1)
};

struct Geo {
    int type, L, N, NB, W;   // W = 32-bit words of packed spins per line (multiple of 4)
    uint64_t magic;          // ceil(2^40 / L): x / L == (x * magic) >> 40 for x < 2^24
    int lshift;              // log2(L) when L is a power of two
    uint32_t lmask;          // L - 1 when L is a power of two
};

// Everything a walker launch needs.  Pointers are device memory.
struct WalkArgs {
    Geo g;
    const LineDesc* desc;
    LineState* st;
    void* perm;              // lines x pstride list entries (uint16 if N <= 65536, else uint32)
    uint32_t* spins;         // lines x W packed spins
    int64_t* lng;            // ragged ln g / u
    hist_t* hist;            // ragged histogram | kVisited
    const uint32_t* table;   // exp threshold table (kTableN words)
    const int32_t* order;    // work queue: line indices, most expensive first
    int32_t* qnext;          // work queue head
    int32_t nqueue;
    int32_t q;               // table shift
    float seg_per_log2;      // ln 2 / (2^q u): table segments per halving of exp(-u d)
    float inv_u;             // 1 / u, production acceptance
    uint32_t seed;
    int32_t flat_pm;         // flatness fraction x in 1/1000
    int32_t stage_smem;      // 1: lists and spins staged in shared memory
    int32_t slot_bytes;      // shared bytes per walker slot (window + staged list/spins)
    int32_t pstride;         // list entries per line, N rounded up to 16 bytes
    int32_t same_f_resets;   // R > 0: extra histogram resets at unchanged f (see walk_line)
    int32_t tbl_mask;        // conflict filter table: tbl_mask + 1 words per walker (tail kernel)
    int64_t C;               // flatness check interval
    int64_t C_per_bin;       // > 0: a line of n bins checks every max(C, C_per_bin * n) moves
    int64_t budget;          // per-line cap on t
    int64_t slice_moves;     // moves per line in this launch
    const uint64_t* deadline_ns;      // device globaltimer deadline (0 = none), may be null
    const uint64_t* slice_end_ns;     // end of this slice in device time (0 = none), may be null
    const volatile int32_t* abort_flag;   // host-mapped stop request, may be null
    int32_t* flags;          // device flags: bit0 deadline, bit1 aborted, bit2 overflow, bit3 invariant
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products on
// words 0 and 2 with the state rearranged as (hi1^c1^k0, lo1, hi0^c3^k1, lo0);
// the key advances by the Weyl increments after every round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Index in [0, n) from a 32-bit word: floor(r * n / 2^32).
__device__ __forceinline__ uint32_t pick(uint32_t r, uint32_t n) { return __umulhi(r, n); }

__device__ __forceinline__ uint32_t divL(const Geo& g, uint32_t x)
{
    return (uint32_t)(((uint64_t)x * g.magic) >> 40);
}

__device__ __forceinline__ uint32_t spin_at(const uint32_t* sp, uint32_t n)
{
    return (sp[n >> 5] >> (n & 31u)) & 1u;
}

// Neighbours of site i on the periodic lattice LAT (same rule as wl.h).
template <int LAT>
__device__ __forceinline__ void neighbours(const Geo& g, uint32_t i, uint32_t* nb)
{
    const uint32_t L = (uint32_t)g.L;
    if (LAT == kSquareP2) {
        const uint32_t x = i & g.lmask, yrow = i & ~g.lmask;
        const uint32_t rowL = (uint32_t)g.N - L;      // offset of the last row
        nb[0] = yrow | ((x + 1) & g.lmask);
        nb[1] = yrow | ((x - 1) & g.lmask);
        nb[2] = (yrow == rowL ? 0u : yrow + L) | x;
        nb[3] = (yrow == 0u ? rowL : yrow - L) | x;
    } else if (LAT == kCubic) {
        const uint32_t r = divL(g, i), x = i - r * L;
        const uint32_t zc = divL(g, r), y = r - zc * L;
        const uint32_t xp = x + 1 == L ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
        const uint32_t yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
        const uint32_t zp = zc + 1 == L ? 0 : zc + 1, zm = zc == 0 ? L - 1 : zc - 1;
        const uint32_t row = (zc * L + y) * L;
        nb[0] = row + xp;
        nb[1] = row + xm;
        nb[2] = (zc * L + yp) * L + x;
        nb[3] = (zc * L + ym) * L + x;
        nb[4] = (zp * L + y) * L + x;
        nb[5] = (zm * L + y) * L + x;
    } else {
        const uint32_t y = divL(g, i), x = i - y * L;
        const uint32_t xp = x + 1 == L ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
        const uint32_t yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
        nb[0] = y * L + xp;
        nb[1] = y * L + xm;
        nb[2] = yp * L + x;
        nb[3] = ym * L + x;
        if (LAT == kTriangular) {
            nb[4] = ym * L + xp;
            nb[5] = yp * L + xm;
        }
    }
}

template <int LAT> struct Coord {
    static constexpr int z = (LAT == kSquare || LAT == kSquareP2 || LAT == kSquareOpen) ? 4 : 6;
    static constexpr int kshift = LAT == kSquareOpen ? 0 : 1;   // bin of k = k >> kshift
    static constexpr int zbin = (2 * z) >> kshift;                // largest bin step of a move
};

// Open boundaries: the neighbours that exist get their index, the others the
// site itself with a cleared valid bit.
__device__ __forceinline__ unsigned open_neighbours(const Geo& g, uint32_t i, uint32_t* nb)
{
    const uint32_t L = (uint32_t)g.L;
    const uint32_t y = divL(g, i), x = i - y * L;
    const unsigned v = (x + 1 < L ? 1u : 0u) | (x > 0 ? 2u : 0u) | (y + 1 < L ? 4u : 0u) | (y > 0 ? 8u : 0u);
    nb[0] = (v & 1u) ? i + 1 : i;
    nb[1] = (v & 2u) ? i - 1 : i;
    nb[2] = (v & 4u) ? i + L : i;
    nb[3] = (v & 8u) ? i - L : i;
    return v;
}

// delta_k that also returns the neighbour lists of i and j (used to decide
// which later proposals an accepted exchange of i and j can affect).
template <int LAT>
__device__ __forceinline__ int delta_k_nb(const Geo& g, const uint32_t* sp, uint32_t i, uint32_t j,
                                          uint32_t* ni, uint32_t* nj)
{
    constexpr int z = Coord<LAT>::z;
    if constexpr (LAT == kSquareOpen) {
        // with degrees z_i, z_j: dk = 2 (u_i - u_j + a_ij) - z_i + z_j
        const unsigned vi = open_neighbours(g, i, ni), vj = open_neighbours(g, j, nj);
        int ui = 0, uj = 0, a = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            ui += (int)(((vi >> m) & 1u) & spin_at(sp, ni[m]));
            uj += (int)(((vj >> m) & 1u) & spin_at(sp, nj[m]));
            a += (int)(((vi >> m) & 1u) && ni[m] == j);
            if (!((vi >> m) & 1u)) ni[m] = 0xFFFFFFFFu;     // never equal to a site
            if (!((vj >> m) & 1u)) nj[m] = 0xFFFFFFFFu;
        }
        return 2 * (ui - uj + a) - __popc(vi) + __popc(vj);
    }
    neighbours<LAT>(g, i, ni);
    neighbours<LAT>(g, j, nj);
    int ui = 0, uj = 0, a = 0;
#pragma unroll
    for (int m = 0; m < z; ++m) {
        ui += (int)spin_at(sp, ni[m]);
        uj += (int)spin_at(sp, nj[m]);
        a += (int)(ni[m] == j);
    }
    return 2 * (ui - uj + a);
}

// Eq. 3 as a threshold on d, the ln g difference g(k')/g(k) in units of u.
// Both acceptance rules are non-increasing in d, so the uphill moves a random
// word r accepts are d = 1 .. dmax(r), and a move is accepted iff d <= dmax(r)
// (every d <= 0 is accepted: dmax >= 0).  dmax depends on the random word
// only, so it is computed when the word is drawn, ahead of the walk.
//
// Deterministic rule: accept iff r < T(d), T the linear interpolation of the
// 4096-entry table t[i] = round(2^32 exp(-i 2^q u)) (t[0] = 2^32 implicit,
// T = 0 from d = 4095 * 2^q on).  With i* the last segment whose left entry is
// above r, the accepted d of that segment are those with
//     (t0 - t1) * frac >> q  <  t0 - r,
// a bound on frac solved exactly in integers below.  i* is first estimated
// from the exponential form of the table and then confirmed (or walked to)
// by integer comparisons, so the result never depends on the estimate.
__device__ __forceinline__ uint64_t table_at(const uint32_t* tab, int i)
{
    return i == 0 ? (1ull << 32) : (uint64_t)tab[i];
}

// Rare path of dmax_det: the segment by bisection (t[lo] > r >= t[hi]).
static __device__ __noinline__ int dmax_segment_search(uint32_t r, const uint32_t* tab)
{
    int lo = 0, hi = kTableN - 1;
    if (table_at(tab, hi - 1) > (uint64_t)r) return hi - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (table_at(tab, mid) > (uint64_t)r) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Integer <-> float conversions by bit manipulation (the 64-bit conversion
// instructions run on the FP64 pipe, which is slow on this GPU).
// u64 -> float, mantissa truncated (relative error below 2^-23).
__device__ __forceinline__ float u64_to_float_rz(uint64_t x)
{
    if (x == 0) return 0.0f;
    const int lz = __clzll((long long)x);
    const uint32_t m = (uint32_t)((x << lz) >> 40);          // 24 bits, top bit set
    return __uint_as_float(((uint32_t)(190 - lz) << 23) | (m & 0x7FFFFFu));
}

// floor of a float in [0, 2^62]
__device__ __forceinline__ int64_t float_floor_i64(float f)
{
    const uint32_t bits = __float_as_uint(f);
    const int e = (int)(bits >> 23) - 127;                   // f = 1.m * 2^e
    if (e < 0) return 0;
    const uint64_t m = (bits & 0x7FFFFFu) | 0x800000u;
    return e >= 23 ? (int64_t)(m << (e - 23)) : (int64_t)(m >> (23 - e));
}

__device__ __forceinline__ int64_t dmax_det(uint32_t r, const uint32_t* tab, int q, float seg_per_log2)
{
    // t[i] ~ 2^32 * 2^(-i / seg_per_log2)  =>  i* ~ (32 - log2 r) * seg_per_log2;
    // the segment is one of c-1, c, c+1 unless r is tiny (the table's flat tail)
    const uint32_t r1 = r | 1u;
    const int lz = __clz(r1);
    const uint32_t frac = (uint32_t)(((uint64_t)r1 << (lz + 1)) >> 9) & 0x7FFFFFu;   // bits below the leading one
    const float lr = __log2f(__uint_as_float(0x3F800000u | frac)) + (float)(31 - lz);
    int c = (int)float_floor_i64(fmaxf((32.0f - lr) * seg_per_log2, 0.0f));
    c = c < 1 ? 1 : (c > kTableN - 3 ? kTableN - 3 : c);
    const uint64_t R = r;
    const uint64_t tm = table_at(tab, c - 1), t0 = (uint64_t)tab[c], t1 = (uint64_t)tab[c + 1],
                   t2 = (uint64_t)tab[c + 2];
    // i* = max{i <= 4094 : t[i] > r}, t non-increasing
    int seg;
    uint64_t a, b;                  // t[i*], t[i*+1]
    if (t0 > R && t1 <= R) {
        seg = c; a = t0; b = t1;
    } else if (tm > R && t0 <= R) {
        seg = c - 1; a = tm; b = t0;
    } else if (t1 > R && (t2 <= R || c + 1 == kTableN - 2)) {
        seg = c + 1; a = t1; b = t2;
    } else {
        seg = dmax_segment_search(r, tab);
        a = table_at(tab, seg);
        b = table_at(tab, seg + 1);
    }
    if (b > R) return ((int64_t)(kTableN - 1) << q) - 1;   // the whole last segment
    // largest frac < 2^q with diff * frac < X 2^q, i.e. floor((X 2^q - 1) / diff)
    const uint64_t X = a - R;                 // 1 .. diff
    const uint32_t diff = (uint32_t)(a - b);  // < 2^32
    const uint64_t num = (X << q) - 1ull;
    float rd;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd) : "f"(u64_to_float_rz(diff)));
    int64_t fr = float_floor_i64(u64_to_float_rz(num) * rd);
    // the float quotient is within a unit or two up to q = 22; exact steps finish it
    while (fr > 0 && (uint64_t)diff * (uint64_t)fr > num) --fr;
    while ((uint64_t)diff * (uint64_t)(fr + 1) <= num) ++fr;
    return ((int64_t)seg << q) + fr;
}

// Production rule: accept iff U < exp(-u d), U = (r/2^8 + 1/2) 2^-24 in (0, 1),
// i.e. d < -ln(U) / u; dmax = floor of that bound (FP32).  Near U = 1 the
// logarithm is taken of 1 - U, which is exact in FP32 there.
__device__ __forceinline__ int64_t dmax_prod(uint32_t r, float inv_u)
{
    const uint32_t mm = r >> 8;
    const float nl = mm >= (1u << 23) ? -log1pf(-((float)((1u << 24) - mm) - 0.5f) * 0x1p-24f)
                                      : -__logf(((float)mm + 0.5f) * 0x1p-24f);
    return float_floor_i64(fminf(nl * inv_u, 0x1p62f));
}

// The random numbers of one move attempt, drawn ahead of the walk: list slots
// a (of the l up spins) and b (of the N - l down spins) and dmax of Eq. 3.
struct Draw {
    uint32_t a, b;
    int64_t dmax;
};

// ---------------------------------------------------------------------------
// Group helpers: S consecutive lanes of a warp serve one walker.
// ---------------------------------------------------------------------------
template <int S, typename T>
__device__ __forceinline__ T group_sum(unsigned gmask, T v)
{
#pragma unroll
    for (int off = S / 2; off > 0; off >>= 1) v += __shfl_xor_sync(gmask, v, off);
    return v;
}

template <int S>
__device__ __forceinline__ int64_t group_min(unsigned gmask, int64_t v)
{
#pragma unroll
    for (int off = S / 2; off > 0; off >>= 1) {
        const int64_t o = __shfl_xor_sync(gmask, v, off);
        v = o < v ? o : v;
    }
    return v;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace wl

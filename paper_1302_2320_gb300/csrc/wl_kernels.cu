// wl_kernels.cu -- walker initialisation, DOS assembly, the device-built exp
// threshold table, the Philox check kernel and the per-launch run summary.
#include <cfloat>
#include <cmath>

#include "wl_kernels.cuh"

namespace wl {

// ---------------------------------------------------------------------------
// Walker initialisation (the initial state of the text around Eq. 3): one warp
// per line.  l up spins at the sites perm[0, l) of a partial Fisher-Yates
// shuffle (step t swaps perm[t] with perm[t + pick(r.x, N - t)], r = Philox
// counter (t, 0, 1, 0), key (l, seed)); U = perm[0, l), D = perm[l, N); ln g = 0,
// h = 0, ln f = 1 (F0 = round(1/u)); k0 counted from the spins.  The line l = 0
// has no exchange move: its single bin k = 0 is marked visited and it is done.
// ---------------------------------------------------------------------------
template <int LAT, typename IDX>
__global__ void init_kernel(const InitArgs A)
{
    const int warps = blockDim.x >> 5;
    const int li = blockIdx.x * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (li >= A.nlines) return;
    const LineDesc D = A.desc[li];
    const int N = A.g.N, W = A.g.W, ell = D.ell;
    IDX* perm = reinterpret_cast<IDX*>(A.perm) + (size_t)li * A.pstride;
    uint32_t* sp = A.spins + (size_t)li * W;
    int64_t* lng = A.lng + D.bin_off;
    hist_t* hist = A.hist + D.bin_off;
    for (int n = lane; n < A.pstride; n += 32) perm[n] = (IDX)(n < N ? n : 0);
    for (int w = lane; w < W; w += 32) sp[w] = 0u;
    for (int b = lane; b < D.nbins; b += 32) {
        lng[b] = 0;
        hist[b] = 0ull;
    }
    __syncwarp();
    const uint2 key = make_uint2((uint32_t)ell, A.seed);
    const int tmax = ell < N - 1 ? ell : N - 1;
    for (int base = 0; base < tmax; base += 32) {
        const int t = base + lane;
        uint32_t j = 0;
        if (t < tmax) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)t, 0u, 1u, 0u), key);
            j = (uint32_t)t + pick(r.x, (uint32_t)(N - t));
        }
        const int cnt = tmax - base < 32 ? tmax - base : 32;
        for (int s = 0; s < cnt; ++s) {
            const uint32_t js = __shfl_sync(0xffffffffu, j, s);
            if (lane == 0) {
                const IDX x = perm[base + s];
                perm[base + s] = perm[js];
                perm[js] = x;
            }
        }
        __syncwarp();
    }
    for (int a = lane; a < ell; a += 32) {
        const uint32_t n = (uint32_t)perm[a];
        atomicOr(&sp[n >> 5], 1u << (n & 31u));
    }
    __syncwarp();
    int twice = 0;
    constexpr int z = Coord<LAT>::z;
    for (int n = lane; n < N; n += 32) {
        uint32_t nb[z];
        unsigned valid = (1u << z) - 1u;
        if constexpr (LAT == kSquareOpen) valid = open_neighbours(A.g, (uint32_t)n, nb);
        else neighbours<LAT>(A.g, (uint32_t)n, nb);
        const uint32_t sn = spin_at(sp, (uint32_t)n);
#pragma unroll
        for (int m = 0; m < z; ++m) twice += (int)(((valid >> m) & 1u) && sn != spin_at(sp, nb[m]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) twice += __shfl_xor_sync(0xffffffffu, twice, off);
    if (lane == 0) {
        LineState s;
        s.k = twice / 2;
        s.t = 0;
        s.F = A.F0;
        s.stage = 0;
        s.accepts = 0;
        s.t_stage = 0;
        s.status = 0;
        s.checks = 0;
        s.batches = 0;
        if (ell == 0) {
            hist[s.k >> Coord<LAT>::kshift] = kVisited;
            s.F = 0;
            s.status = 1;
        }
        A.st[li] = s;
    }
}

cudaError_t launch_init(int lattice, bool idx16, const InitArgs& a, cudaStream_t s)
{
    clear_stale_error();
    const int warps = 4;
    const dim3 grid((a.nlines + warps - 1) / warps), block(32 * warps);
    if (lattice == kSquare) {
        if (idx16) init_kernel<kSquare, uint16_t><<<grid, block, 0, s>>>(a);
        else init_kernel<kSquare, uint32_t><<<grid, block, 0, s>>>(a);
    } else if (lattice == kTriangular) {
        if (idx16) init_kernel<kTriangular, uint16_t><<<grid, block, 0, s>>>(a);
        else init_kernel<kTriangular, uint32_t><<<grid, block, 0, s>>>(a);
    } else if (lattice == kCubic) {
        if (idx16) init_kernel<kCubic, uint16_t><<<grid, block, 0, s>>>(a);
        else init_kernel<kCubic, uint32_t><<<grid, block, 0, s>>>(a);
    } else {
        if (idx16) init_kernel<kSquareOpen, uint16_t><<<grid, block, 0, s>>>(a);
        else init_kernel<kSquareOpen, uint32_t><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Assembly (Eq. 4 applied once, g_kl of Eq. 2): one warp per line,
//   ln g_kl = ln C(N,l) + u lng[b] - (M + ln sum_visited exp(u lng[b] - M)),
// M the visited maximum; unvisited bins get -inf.  FP64.
// ---------------------------------------------------------------------------
__global__ void assemble_kernel(const LineDesc* desc, const int64_t* lng, const hist_t* hist,
                                int N, int nlines, double u, double* out)
{
    const int warps = blockDim.x >> 5;
    const int li = blockIdx.x * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (li >= nlines) return;
    const LineDesc D = desc[li];
    const int64_t* lg = lng + D.bin_off;
    const hist_t* h = hist + D.bin_off;
    double* o = out + D.bin_off;
    double mx = -DBL_MAX;
    for (int b = lane; b < D.nbins; b += 32)
        if (h[b] & kVisited) mx = fmax(mx, u * (double)lg[b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    double sum = 0.0;
    for (int b = lane; b < D.nbins; b += 32)
        if (h[b] & kVisited) sum += exp(u * (double)lg[b] - mx);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    const double lse = mx + log(sum);
    const double lnC = lgamma((double)N + 1.0) - lgamma((double)D.ell + 1.0) -
                       lgamma((double)(N - D.ell) + 1.0);
    for (int b = lane; b < D.nbins; b += 32)
        o[b] = (h[b] & kVisited) ? lnC + u * (double)lg[b] - lse : -INFINITY;
}

cudaError_t launch_assemble(const LineDesc* desc, const int64_t* lng, const hist_t* hist, int N,
                            int nlines, double u, double* out, cudaStream_t s)
{
    clear_stale_error();
    const int warps = 8;
    assemble_kernel<<<(nlines + warps - 1) / warps, 32 * warps, 0, s>>>(desc, lng, hist, N, nlines,
                                                                       u, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exp threshold table, built on the device: t[i] = floor(2^32 exp(-x_i) + 1/2),
// x_i = (i 2^q) u as one IEEE double product.  exp is evaluated in
// double-double arithmetic (Dekker's exact products and sums): x = n ln2 + r
// with ln 2 split in two doubles, exp(r / 2^10) by its Taylor series to degree
// 10, then ten squarings; relative error ~1e-28, far below the 2^-33
// granularity of the rounding.
// ---------------------------------------------------------------------------
struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dd dd_norm(double a, double b)
{
    const double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}

__device__ __forceinline__ dd dd_add(dd a, dd b)
{
    dd s = dd_two_sum(a.hi, b.hi);
    const dd t = dd_two_sum(a.lo, b.lo);
    s.lo = __dadd_rn(s.lo, t.hi);
    s = dd_norm(s.hi, s.lo);
    s.lo = __dadd_rn(s.lo, t.lo);
    return dd_norm(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_mul(dd a, dd b)
{
    const double p = __dmul_rn(a.hi, b.hi);
    double e = __fma_rn(a.hi, b.hi, -p);
    e = __fma_rn(a.hi, b.lo, e);
    e = __fma_rn(a.lo, b.hi, e);
    return dd_norm(p, e);
}

__device__ __forceinline__ dd dd_mul_d(dd a, double b)
{
    const double p = __dmul_rn(a.hi, b);
    const double e = __fma_rn(a.lo, b, __fma_rn(a.hi, b, -p));
    return dd_norm(p, e);
}

__device__ dd dd_exp_neg(double x)   // exp(-x) for 0 <= x < 40
{
    const dd ln2 = {0x1.62e42fefa39efp-1, 0x1.abc9e3b39803fp-56};
    const double n = rint(x / ln2.hi);
    // r = n ln2 - x  (exact enough: |r| <= 0.35)
    dd r = dd_mul_d(ln2, n);
    r = dd_add(r, {-x, 0.0});
    r.hi = ldexp(r.hi, -10);
    r.lo = ldexp(r.lo, -10);
    // Taylor series of exp(r) - 1, Horner form: r (1 + r/2 (1 + r/3 (...)))
    dd s = {1.0, 0.0};
    for (int k = 10; k >= 1; --k) {
        dd term = dd_mul(s, r);
        // divide by k: term / k in double-double via multiplication by 1/k corrections
        const double qh = __ddiv_rn(term.hi, (double)k);
        const double rem = __fma_rn(-qh, (double)k, term.hi);
        const double ql = __ddiv_rn(__dadd_rn(rem, term.lo), (double)k);
        s = dd_add({1.0, 0.0}, dd_norm(qh, ql));
    }
    // s = exp(r); square ten times
    for (int k = 0; k < 10; ++k) s = dd_mul(s, s);
    // times 2^-n
    s.hi = ldexp(s.hi, -(int)n);
    s.lo = ldexp(s.lo, -(int)n);
    return s;
}

__global__ void exp_table_kernel(double u, int q, uint64_t* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kTableN) return;
    const double x = __dmul_rn((double)((uint64_t)i << q), u);
    dd e = dd_exp_neg(x);
    // v = 2^32 e + 1/2, floor(v) with v = hi + lo
    const double hi = ldexp(e.hi, 32), lo = ldexp(e.lo, 32);
    const double fh = floor(hi);
    const double frac = __dadd_rn(__dadd_rn(__dsub_rn(hi, fh), lo), 0.5);
    out[i] = (uint64_t)fh + (uint64_t)floor(frac);
}

cudaError_t launch_exp_table(double u, int q, uint64_t* out, cudaStream_t s)
{
    clear_stale_error();
    exp_table_kernel<<<(kTableN + 255) / 256, 256, 0, s>>>(u, q, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Philox check kernel: one block per counter.
// ---------------------------------------------------------------------------
__global__ void philox_kernel(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
    const uint4 r = philox4x32_10(c, k);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

cudaError_t launch_philox(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    clear_stale_error();
    philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, ctr, key, out);
    return cudaGetLastError();
}

// dmax of Eq. 3 (the walker's acceptance threshold on d) for n random words.
__global__ void dmax_kernel(size_t n, const uint32_t* r, int det, const uint32_t* tab, int q,
                            float seg_per_log2, float inv_u, int64_t* out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = det ? dmax_det(r[i], tab, q, seg_per_log2) : dmax_prod(r[i], inv_u);
}

cudaError_t launch_dmax(size_t n, const uint32_t* r, int det, const uint32_t* tab, int q,
                        float seg_per_log2, float inv_u, int64_t* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    clear_stale_error();
    dmax_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, r, det, tab, q, seg_per_log2, inv_u, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Run summary after each walker launch: one block reduces the line states.
// ---------------------------------------------------------------------------
__global__ void summary_kernel(const LineState* st, int nlines, int64_t budget,
                               const int32_t* flags, Summary* out)
{
    __shared__ long long s_moves[32], s_acc[32], s_chk[32], s_bat[32];
    __shared__ int s_active[32], s_conv[32], s_ovf[32], s_min[32], s_max[32];
    long long moves = 0, acc = 0, chk = 0, bat = 0;
    int active = 0, conv = 0, ovf = 0, mn = INT_MAX, mx = 0;
    for (int i = threadIdx.x; i < nlines; i += blockDim.x) {
        const LineState s = st[i];
        moves += s.t;
        acc += s.accepts;
        chk += s.checks;
        bat += s.batches;
        active += (s.status == 0 && s.t < budget);
        conv += (s.status == 1);
        ovf += (s.status == 2);
        mn = (int)s.stage < mn ? (int)s.stage : mn;
        mx = (int)s.stage > mx ? (int)s.stage : mx;
    }
    for (int off = 16; off > 0; off >>= 1) {
        moves += __shfl_xor_sync(0xffffffffu, moves, off);
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
        chk += __shfl_xor_sync(0xffffffffu, chk, off);
        bat += __shfl_xor_sync(0xffffffffu, bat, off);
        active += __shfl_xor_sync(0xffffffffu, active, off);
        conv += __shfl_xor_sync(0xffffffffu, conv, off);
        ovf += __shfl_xor_sync(0xffffffffu, ovf, off);
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_moves[w] = moves;
        s_acc[w] = acc;
        s_chk[w] = chk;
        s_bat[w] = bat;
        s_active[w] = active;
        s_conv[w] = conv;
        s_ovf[w] = ovf;
        s_min[w] = mn;
        s_max[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Summary r = {0, 0, 0, 0, 0, 0, 0, INT_MAX, 0, 0};
        for (int x = 0; x < (int)(blockDim.x >> 5); ++x) {
            r.moves += s_moves[x];
            r.accepts += s_acc[x];
            r.checks += s_chk[x];
            r.batches += s_bat[x];
            r.active += s_active[x];
            r.converged += s_conv[x];
            r.overflow += s_ovf[x];
            r.min_stage = min(r.min_stage, s_min[x]);
            r.max_stage = max(r.max_stage, s_max[x]);
        }
        r.flags = *flags;
        *out = r;
    }
}

cudaError_t launch_summary(const LineState* st, int nlines, int64_t budget, const int32_t* flags,
                           Summary* out, cudaStream_t s)
{
    clear_stale_error();
    summary_kernel<<<1, 1024, 0, s>>>(st, nlines, budget, flags, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Thermodynamics from the assembled surface (Eq. 2 with the energy of Eq. 1):
// one block per (T, H) point, Z = sum_{k,l} g_kl exp(-E_kl / T),
// E_kl = -(N_B - 2k) - H M, M = 2l - N; line l > N/2 is line N - l.  A single
// pass keeps an online log-sum-exp (running maximum, sums rescaled when it
// grows) of the weights and of the weighted E, E^2, M, |M|, M^2; FP64.
// ---------------------------------------------------------------------------
struct ThermoAcc {
    double mx, z, e1, e2, m1, ma, m2;
};

__device__ __forceinline__ void thermo_add(ThermoAcc& a, double x, double E, double M)
{
    if (x > a.mx) {
        const double r = exp(a.mx - x);
        a.z *= r; a.e1 *= r; a.e2 *= r; a.m1 *= r; a.ma *= r; a.m2 *= r;
        a.mx = x;
    }
    const double w = exp(x - a.mx);
    a.z += w;
    a.e1 += w * E;
    a.e2 += w * E * E;
    a.m1 += w * M;
    a.ma += w * fabs(M);
    a.m2 += w * M * M;
}

__device__ __forceinline__ void thermo_merge(ThermoAcc& a, const ThermoAcc& b)
{
    if (b.mx == -INFINITY) return;
    if (a.mx == -INFINITY) {
        a = b;
        return;
    }
    const double m = fmax(a.mx, b.mx), ra = exp(a.mx - m), rb = exp(b.mx - m);
    a.z = a.z * ra + b.z * rb;
    a.e1 = a.e1 * ra + b.e1 * rb;
    a.e2 = a.e2 * ra + b.e2 * rb;
    a.m1 = a.m1 * ra + b.m1 * rb;
    a.ma = a.ma * ra + b.ma * rb;
    a.m2 = a.m2 * ra + b.m2 * rb;
    a.mx = m;
}

__device__ __forceinline__ ThermoAcc shfl_acc(const ThermoAcc& a, int off)
{
    ThermoAcc b;
    b.mx = __shfl_xor_sync(0xffffffffu, a.mx, off);
    b.z = __shfl_xor_sync(0xffffffffu, a.z, off);
    b.e1 = __shfl_xor_sync(0xffffffffu, a.e1, off);
    b.e2 = __shfl_xor_sync(0xffffffffu, a.e2, off);
    b.m1 = __shfl_xor_sync(0xffffffffu, a.m1, off);
    b.ma = __shfl_xor_sync(0xffffffffu, a.ma, off);
    b.m2 = __shfl_xor_sync(0xffffffffu, a.m2, off);
    return b;
}

__global__ void thermo_kernel(const LineDesc* desc, int nlines, const double* lng, int N, int NB,
                              int kstep, const double* T, const double* H, int nH, double* out)
{
    const int pt = blockIdx.x;
    const double beta = 1.0 / T[pt / nH], h = H[pt % nH];
    ThermoAcc acc = {-INFINITY, 0, 0, 0, 0, 0, 0};
    for (int li = 0; li < nlines; ++li) {
        const LineDesc D = desc[li];
        const int l = D.ell, lm = N - D.ell;
        const double Mp = (double)(2 * l - N), Mm = (double)(2 * lm - N);
        for (int b = threadIdx.x; b < D.nbins; b += blockDim.x) {
            const double g = lng[D.bin_off + b];
            if (isinf(g)) continue;
            const double bond = -(double)(NB - 2 * kstep * b);       // k = kstep * b
            const double Ep = bond - h * Mp;
            thermo_add(acc, g - beta * Ep, Ep, Mp);
            if (lm != l) {
                const double Em = bond - h * Mm;
                thermo_add(acc, g - beta * Em, Em, Mm);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) thermo_merge(acc, shfl_acc(acc, off));
    __shared__ ThermoAcc part[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) part[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        ThermoAcc a = part[0];
        for (int x = 1; x < (int)(blockDim.x >> 5); ++x) thermo_merge(a, part[x]);
        const double e1 = a.e1 / a.z, e2 = a.e2 / a.z, m1 = a.m1 / a.z, ma = a.ma / a.z,
                     m2 = a.m2 / a.z;
        double* o = out + (size_t)pt * 6;
        o[0] = (a.mx + log(a.z)) / N;
        o[1] = e1 / N;
        o[2] = (e2 - e1 * e1) * beta * beta / N;
        o[3] = m1 / N;
        o[4] = ma / N;
        o[5] = (m2 - m1 * m1) * beta / N;
    }
}

cudaError_t launch_thermo(const LineDesc* desc, int nlines, const double* lng, int N, int NB,
                          int kstep, const double* T, int nT, const double* H, int nH, double* out,
                          cudaStream_t s)
{
    if (nT * nH == 0) return cudaSuccess;
    clear_stale_error();
    thermo_kernel<<<nT * nH, 256, 0, s>>>(desc, nlines, lng, N, NB, kstep, T, H, nH, out);
    return cudaGetLastError();
}

__global__ void deadline_kernel(uint64_t* deadline, uint64_t timeout_ns)
{
    *deadline = timeout_ns ? globaltimer_ns() + timeout_ns : 0ull;
}

cudaError_t launch_set_deadline(uint64_t* deadline, uint64_t timeout_ns, cudaStream_t s)
{
    clear_stale_error();
    deadline_kernel<<<1, 1, 0, s>>>(deadline, timeout_ns);
    return cudaGetLastError();
}

cudaError_t launch_walk(int lattice, int S, bool det, bool idx16, dim3 grid, dim3 block,
                        size_t smem, cudaStream_t s, const WalkArgs& a)
{
    if (lattice == kSquare) return launch_walk_square(S, det, idx16, grid, block, smem, s, a, nullptr);
    if (lattice == kSquareP2)
        return launch_walk_square_p2(S, det, idx16, grid, block, smem, s, a, nullptr);
    if (lattice == kTriangular)
        return launch_walk_triangular(S, det, idx16, grid, block, smem, s, a, nullptr);
    if (lattice == kSquareOpen)
        return launch_walk_square_open(S, det, idx16, grid, block, smem, s, a, nullptr);
    return launch_walk_cubic(S, det, idx16, grid, block, smem, s, a, nullptr);
}

cudaError_t walk_kernel_attrs(int lattice, int S, bool det, bool idx16, size_t smem,
                              int block_threads, int* blocks_per_sm, bool tbl)
{
    WalkArgs dummy{};
    dummy.tbl_mask = tbl ? 1 : 0;
    const dim3 z(0), b(block_threads);
    if (lattice == kSquare) return launch_walk_square(S, det, idx16, z, b, smem, 0, dummy, blocks_per_sm);
    if (lattice == kSquareP2)
        return launch_walk_square_p2(S, det, idx16, z, b, smem, 0, dummy, blocks_per_sm);
    if (lattice == kTriangular)
        return launch_walk_triangular(S, det, idx16, z, b, smem, 0, dummy, blocks_per_sm);
    if (lattice == kSquareOpen)
        return launch_walk_square_open(S, det, idx16, z, b, smem, 0, dummy, blocks_per_sm);
    return launch_walk_cubic(S, det, idx16, z, b, smem, 0, dummy, blocks_per_sm);
}

}  // namespace wl

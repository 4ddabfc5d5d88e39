// mh.cu -- the local Metropolis-Hastings comparator of Sec. 4 on the GPU:
// checkerboard sweeps of single-spin-flip proposals over many chains, to set
// the cost of a sweep against the cost of an HMC trajectory.
//
// Spins are int8 (+-1), chain-major, or, when rows are a multiple of 32 long,
// packed 32 per word (multi-spin coding, mh_packed_kernel).  A sweep is three launches: colour 0,
// colour 1 (c = (x + y + z) mod 2; with every extent even each bond joins the
// two colours, so the sites of one colour see only the other colour and are
// updated in parallel with the result of any sequential order), then a
// per-chain step that turns the sweep's integer sums into observables.  A
// thread owns 8 consecutive sites (group q; one 8-byte word when rows are a
// multiple of 8 long), draws one Philox block per
// half-sweep for the 4 of them that have its colour (site i uses word
// (i/2) mod 4 of block i/8), and flips site i iff u23 < p, p from the chain's
// FP32 table of min(1, exp(-2 beta s (J nb + h))) over s and the neighbour sum
// nb.  The colour-0 launch adds its spins to the chain's spin sum M; the
// colour-1 launch adds its spins and s_i * nb_i, which counts every bond once,
// to M and the bond sum B (integers, exact in any order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "device_common.cuh"
#include "internal.h"

using namespace ihmc;

namespace {

constexpr uint32_t PURPOSE_MH = 5;
constexpr int MH_THREADS = 256;
constexpr int MH_TAB = 13;   // neighbour sums -6..6

// Per-chain parameters and sums.
struct MHChain {
    double beta, J, h;
    double sums[ISING_NSUMS];
};

struct MHArgs {
    int8_t *s;
    uint32_t *sw;                   // packed form: 32 spins per word, bit = (s == +1)
    const uint32_t *ttab;           // packed form, per chain: [2][8] thresholds, index (s > 0, count)
    const float *ptab;              // per chain: [2][MH_TAB], index (s > 0, nb + 6)
    unsigned long long *acc;        // per chain: M, B, flips (two's complement)
    MHChain *chains;
    int X, Y, Z;
    int64_t N;
    uint64_t seed;
    uint32_t half;                  // 2 * sweep + colour
    int measure;
};

template <int DIM>
__global__ void __launch_bounds__(MH_THREADS) mh_colour_kernel(MHArgs a, int colour) {
    __shared__ float tab[2 * MH_TAB];
    const int chain = blockIdx.y;
    if (threadIdx.x < 2 * MH_TAB) tab[threadIdx.x] = a.ptab[chain * 2 * MH_TAB + threadIdx.x];
    __syncthreads();
    const int64_t N = a.N;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int8_t *s = a.s + (int64_t)chain * N;
    int dM = 0, dB = 0, dF = 0;
    if (q < (N + 7) / 8) {
        const u32x4 w = philox((uint32_t)q, a.half, (uint32_t)chain, PURPOSE_MH, a.seed);
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
        const int X = a.X, Y = a.Y, Z = a.Z;
        const int64_t i0 = 8 * q;
        const uint32_t i032 = (uint32_t)i0, r = i032 / (uint32_t)X;   // N <= 2^31
        int x = (int)(i032 - r * (uint32_t)X);
        int y = (int)(r % (uint32_t)Y);
        int z = (int)(r / (uint32_t)Y);
        const int64_t XY = (int64_t)X * Y;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t i = i0 + k;
            if (i >= N) break;
            if (((x + y + z) & 1) == colour) {
                int nb = s[x > 0 ? i - 1 : i + X - 1] + s[x + 1 < X ? i + 1 : i - (X - 1)];
                if constexpr (DIM >= 2)
                    nb += s[y > 0 ? i - X : i + (int64_t)(Y - 1) * X] +
                          s[y + 1 < Y ? i + X : i - (int64_t)(Y - 1) * X];
                if constexpr (DIM == 3)
                    nb += s[z > 0 ? i - XY : i + (int64_t)(Z - 1) * XY] +
                          s[z + 1 < Z ? i + XY : i - (int64_t)(Z - 1) * XY];
                int si = s[i];
                const float u = u23(words[(k >> 1) & 3]);
                if (u < tab[(si > 0 ? MH_TAB : 0) + nb + 6]) {
                    si = -si;
                    s[i] = (int8_t)si;
                    ++dF;
                }
                dM += si;
                if (colour == 1) dB += si * nb;
            }
            if (++x == X) {
                x = 0;
                if (++y == Y) {
                    y = 0;
                    ++z;
                }
            }
        }
    }
    // warp sums, one atomic per warp and quantity
    dM = __reduce_add_sync(0xffffffffu, dM);
    dB = __reduce_add_sync(0xffffffffu, dB);
    dF = __reduce_add_sync(0xffffffffu, dF);
    if ((threadIdx.x & 31) == 0) {
        unsigned long long *acc = a.acc + 3 * chain;
        if (dM) atomicAdd(acc + 0, (unsigned long long)(long long)dM);
        if (dB) atomicAdd(acc + 1, (unsigned long long)(long long)dB);
        if (dF) atomicAdd(acc + 2, (unsigned long long)(long long)dF);
    }
}

// Fast path for rows whose length is a multiple of 8: a thread's 8 sites lie in
// one row and are read as one 8-byte word, the rows above and below (and the
// planes in 3D) as 8-byte words too, the two x-neighbours at the ends as
// bytes; flipped sites are stored byte by byte (the other colour's bytes,
// which neighbouring threads are reading, are never written).  The same
// draws, decisions and sums as mh_colour_kernel.
__device__ __forceinline__ int sbyte(uint64_t w, int k) { return (int)(int8_t)(w >> (8 * k)); }

template <int DIM>
__device__ __forceinline__ void row8_group(const MHArgs &a, int colour, int chain, int8_t *s,
                                           const uint64_t *s8, const float *tab, uint32_t q,
                                           int &dM, int &dB, int &dF) {
    const uint32_t X = (uint32_t)a.X, Y = (uint32_t)a.Y, Z = (uint32_t)a.Z;
    const uint32_t X8 = X >> 3;
    const uint32_t row = q / X8;                 // 32-bit index arithmetic: N <= 2^31
    const uint32_t x0 = (q - row * X8) << 3;
    const uint32_t y = row % Y, z = row / Y;
    const uint32_t i0 = q << 3;
    const uint64_t c = s8[q];
    uint64_t ym = 0, yp = 0, zm = 0, zp = 0;
    if constexpr (DIM >= 2) {
        ym = s8[(y > 0 ? i0 - X : i0 + (Y - 1) * X) >> 3];
        yp = s8[(y + 1 < Y ? i0 + X : i0 - (Y - 1) * X) >> 3];
    }
    if constexpr (DIM == 3) {
        const uint32_t XY = X * Y;
        zm = s8[(z > 0 ? i0 - XY : i0 + (Z - 1) * XY) >> 3];
        zp = s8[(z + 1 < Z ? i0 + XY : i0 - (Z - 1) * XY) >> 3];
    }
    const int left = s[x0 > 0 ? i0 - 1 : i0 + X - 1];
    const int right = s[x0 + 8 < X ? i0 + 8 : i0 + 8 - X];
    const u32x4 w = philox(q, a.half, (uint32_t)chain, PURPOSE_MH, a.seed);
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
    const int k0 = (int)((colour + y + z) & 1);   // x0 is even: site k has colour (k + y + z) mod 2
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int k = k0 + 2 * m;
        int nb = (k == 0 ? left : sbyte(c, k - 1)) + (k == 7 ? right : sbyte(c, k + 1));
        if constexpr (DIM >= 2) nb += sbyte(ym, k) + sbyte(yp, k);
        if constexpr (DIM == 3) nb += sbyte(zm, k) + sbyte(zp, k);
        int si = sbyte(c, k);
        if (u23(words[m]) < __ldg(tab + (si > 0 ? MH_TAB : 0) + nb + 6)) {
            si = -si;
            s[i0 + k] = (int8_t)si;
            ++dF;
        }
        dM += si;
        if (colour == 1) dB += si * nb;
    }
}

// Two groups per thread (q and q + half the grid's groups), so each thread
// has two sets of loads in flight.
template <int DIM>
__global__ void __launch_bounds__(MH_THREADS) mh_colour_row8_kernel(MHArgs a, int colour) {
    const int chain = blockIdx.y;
    const uint32_t groups = (uint32_t)(a.N >> 3);
    const uint32_t stride = gridDim.x * blockDim.x;
    int8_t *s = a.s + (int64_t)chain * a.N;
    const uint64_t *s8 = reinterpret_cast<const uint64_t *>(s);
    const float *tab = a.ptab + chain * 2 * MH_TAB;
    int dM = 0, dB = 0, dF = 0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < groups; q += stride)
        row8_group<DIM>(a, colour, chain, s, s8, tab, q, dM, dB, dF);
    dM = __reduce_add_sync(0xffffffffu, dM);
    dB = __reduce_add_sync(0xffffffffu, dB);
    dF = __reduce_add_sync(0xffffffffu, dF);
    if ((threadIdx.x & 31) == 0) {
        unsigned long long *acc = a.acc + 3 * chain;
        if (dM) atomicAdd(acc + 0, (unsigned long long)(long long)dM);
        if (dB) atomicAdd(acc + 1, (unsigned long long)(long long)dB);
        if (dF) atomicAdd(acc + 2, (unsigned long long)(long long)dF);
    }
}

// Multi-spin-coded form, rows a multiple of 32 long: 32 spins of a row per
// 32-bit word (bit j = site x0 + j, set for spin +1).  A thread owns one word:
// the neighbour words give the left/right neighbour bit-vectors by shifts
// (the row's end bits from the adjacent words, periodic), the other
// directions whole words; a bit-sliced adder counts each lane's +1
// neighbours (cnt = (nb + 2 dim) / 2).  The 16 lanes of the launch's colour
// take their decisions with the same Philox words as the byte kernels (site i
// uses word (i/2) mod 4 of block i/8, so lane k0 + 2m uses word m & 3 of block
// 4w + m/4) against an integer threshold: (x >> 9) < T with T the number of
// 23-bit values k with (k + 1/2) 2^-23 < p, i.e. exactly the FP32 test
// u23(x) < p.  Spins, flips and sums equal the byte kernels' bit for bit.
__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
    return (a & b) | (c & (a ^ b));
}

template <int DIM>
__global__ void __launch_bounds__(MH_THREADS) mh_packed_kernel(MHArgs a, int colour) {
    __shared__ uint32_t tt[16];
    const int chain = blockIdx.y;
    if (threadIdx.x < 16) tt[threadIdx.x] = a.ttab[chain * 16 + threadIdx.x];
    __syncthreads();
    const uint32_t X = (uint32_t)a.X, Y = (uint32_t)a.Y, Z = (uint32_t)a.Z;
    const uint32_t XW = X >> 5;                        // words per row
    const uint32_t nw = (uint32_t)(a.N >> 5);          // words per chain
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    int dM = 0, dB = 0, dF = 0;
    if (w < nw) {
        uint32_t *sw = a.sw + (int64_t)chain * nw;
        const uint32_t row = w / XW;                   // 32-bit index arithmetic: N <= 2^31
        const uint32_t xw = w - row * XW;
        const uint32_t y = row % Y, z = row / Y;
        const uint32_t c = sw[w];
        const uint32_t wl = xw > 0 ? w - 1 : w + XW - 1;
        const uint32_t wr = xw + 1 < XW ? w + 1 : w + 1 - XW;
        const uint32_t Lv = (c << 1) | (sw[wl] >> 31);      // lane j: site x - 1
        const uint32_t Rv = (c >> 1) | (sw[wr] << 31);      // lane j: site x + 1
        uint32_t b0, b1, b2 = 0u;
        if constexpr (DIM == 1) {
            b0 = Lv ^ Rv;
            b1 = Lv & Rv;
        } else {
            const uint32_t RW = XW * Y;                // words per plane
            const uint32_t Uv = sw[y > 0 ? w - XW : w + (Y - 1) * XW];
            const uint32_t Dv = sw[y + 1 < Y ? w + XW : w - (Y - 1) * XW];
            if constexpr (DIM == 2) {
                const uint32_t s1 = Lv ^ Rv, c1 = Lv & Rv, s2 = Uv ^ Dv, c2 = Uv & Dv;
                b0 = s1 ^ s2;
                const uint32_t k = s1 & s2;
                b1 = c1 ^ c2 ^ k;
                b2 = maj3(c1, c2, k);
            } else {
                const uint32_t Fv = sw[z > 0 ? w - RW : w + (Z - 1) * RW];
                const uint32_t Bv = sw[z + 1 < Z ? w + RW : w - (Z - 1) * RW];
                const uint32_t s1 = Lv ^ Rv ^ Uv, c1 = maj3(Lv, Rv, Uv);
                const uint32_t s2 = Dv ^ Fv ^ Bv, c2 = maj3(Dv, Fv, Bv);
                b0 = s1 ^ s2;
                const uint32_t k = s1 & s2;
                b1 = c1 ^ c2 ^ k;
                b2 = maj3(c1, c2, k);
            }
        }
        // lanes of this colour: j = k0 + 2m (x0 is a multiple of 32, so even)
        const uint32_t k0 = (uint32_t)(colour + y + z) & 1u;
        const uint32_t e0 = b0 >> k0, e1 = b1 >> k0, e2 = b2 >> k0, es = c >> k0;
        uint32_t fl = 0u;   // flips, lane m at bit 2m
#pragma unroll
        for (int blk = 0; blk < 4; ++blk) {
            const u32x4 r = philox(4 * w + (uint32_t)blk, a.half, (uint32_t)chain, PURPOSE_MH,
                                   a.seed);
            const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = 4 * blk + q, sh = 2 * m;
                const uint32_t idx = ((es >> sh) & 1u) << 3 | ((e2 >> sh) & 1u) << 2 |
                                     ((e1 >> sh) & 1u) << 1 | ((e0 >> sh) & 1u);
                fl |= (uint32_t)((rw[q] >> 9) < tt[idx]) << sh;
            }
        }
        const uint32_t lanes = 0x55555555u << k0;
        const uint32_t flips = fl << k0;
        const uint32_t nc = c ^ flips;
        sw[w] = nc;
        const int up = __popc(nc & lanes);
        dM = 2 * up - 16;
        dF = __popc(flips);
        if (colour == 1) {
            // sum over the lanes of s * nb, nb = 2 cnt - 2 DIM
            const uint32_t pl = nc & lanes, mi = ~nc & lanes;
            const int cp = __popc(b0 & pl) + 2 * __popc(b1 & pl) + 4 * __popc(b2 & pl);
            const int cm = __popc(b0 & mi) + 2 * __popc(b1 & mi) + 4 * __popc(b2 & mi);
            dB = (2 * cp - 2 * DIM * up) - (2 * cm - 2 * DIM * (16 - up));
        }
    }
    dM = __reduce_add_sync(0xffffffffu, dM);
    dB = __reduce_add_sync(0xffffffffu, dB);
    dF = __reduce_add_sync(0xffffffffu, dF);
    if ((threadIdx.x & 31) == 0) {
        unsigned long long *acc = a.acc + 3 * chain;
        if (dM) atomicAdd(acc + 0, (unsigned long long)(long long)dM);
        if (dB) atomicAdd(acc + 1, (unsigned long long)(long long)dB);
        if (dF) atomicAdd(acc + 2, (unsigned long long)(long long)dF);
    }
}

// Observables of the sweep just finished (if measured), then clear the sums.
__global__ void mh_measure_kernel(MHArgs a, int n_chains) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    unsigned long long *acc = a.acc + 3 * c;
    const long long M = (long long)acc[0], B = (long long)acc[1], F = (long long)acc[2];
    acc[0] = acc[1] = acc[2] = 0ull;
    if (!a.measure) return;
    // explicitly rounded operations in the order written (no contraction),
    // so the sums are reproducible bit for bit
    MHChain &ch = a.chains[c];
    const double Nd = (double)a.N;
    const double m = __ddiv_rn((double)M, Nd);
    const double t = __dsub_rn(__dmul_rn(-ch.J, (double)B), __dmul_rn(ch.h, (double)M));
    const double E = __ddiv_rn(__dmul_rn(ch.beta, t), Nd);
    const double m2 = __dmul_rn(m, m);
    double *sm = ch.sums;
    sm[ISING_SUM_NMEAS] = __dadd_rn(sm[ISING_SUM_NMEAS], 1.0);
    sm[ISING_SUM_NACC] = __dadd_rn(sm[ISING_SUM_NACC], __ddiv_rn((double)F, Nd));
    sm[ISING_SUM_M] = __dadd_rn(sm[ISING_SUM_M], m);
    sm[ISING_SUM_M2] = __dadd_rn(sm[ISING_SUM_M2], m2);
    sm[ISING_SUM_E] = __dadd_rn(sm[ISING_SUM_E], E);
    sm[ISING_SUM_E2] = __dadd_rn(sm[ISING_SUM_E2], __dmul_rn(E, E));
    sm[ISING_SUM_ABSM] = __dadd_rn(sm[ISING_SUM_ABSM], fabs(m));
    sm[ISING_SUM_ABSM2] = __dadd_rn(sm[ISING_SUM_ABSM2], m2);
}

thread_local char g_mh_create_err[512];

}  // namespace

struct ising_mh {
    int dim = 0, L[3] = {1, 1, 1};
    int64_t N = 0;
    int n_chains = 0, n_therm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool packed = false;            // rows a multiple of 32: 32 spins per word
    int8_t *s = nullptr;            // byte form: one int8 per spin
    uint32_t *sw = nullptr;         // packed form
    uint32_t *ttab = nullptr;       // packed form: per chain [2][8] thresholds
    float *ptab = nullptr;
    unsigned long long *acc = nullptr;
    MHChain *chains = nullptr;
    int64_t sweep = 0, launches = 0;
    char err[512] = {0};
};

static ising_status mh_fail(ising_mh *h, ising_status st, const char *fmt, ...) {
    char *buf = h ? h->err : g_mh_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

static void mh_free(ising_mh *h) {
    if (h->s) cudaFree(h->s);
    if (h->sw) cudaFree(h->sw);
    if (h->ttab) cudaFree(h->ttab);
    h->sw = nullptr;
    h->ttab = nullptr;
    if (h->ptab) cudaFree(h->ptab);
    if (h->acc) cudaFree(h->acc);
    if (h->chains) cudaFree(h->chains);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->s = nullptr;
    h->ptab = nullptr;
    h->acc = nullptr;
    h->chains = nullptr;
    h->stream = nullptr;
}

// Acceptance probability of flipping spin s with neighbour sum nb, formed in
// FP64 in the stated order (the build disables floating-point contraction in
// host code) and rounded to FP32.
static float accept_prob(double beta, double J, double h, int s, int nb) {
    double f = J * (double)nb + h;
    double x = -2.0 * beta * (double)s * f;
    double p = x >= 0.0 ? 1.0 : std::exp(x);
    return (float)p;
}

// Number of 23-bit values k with (k + 1/2) 2^-23 < p: the packed kernel's
// integer test (x >> 9) < T equals the FP32 test u23(x) < p exactly (p and
// p 2^23 are exact in FP64).
static uint32_t accept_threshold(float p) {
    const double t = std::ceil((double)p * 8388608.0 - 0.5);
    return t <= 0.0 ? 0u : t >= 8388608.0 ? 8388608u : (uint32_t)t;
}

static MHArgs mh_args(ising_mh *h) {
    MHArgs a{};
    a.s = h->s;
    a.sw = h->sw;
    a.ttab = h->ttab;
    a.ptab = h->ptab;
    a.acc = h->acc;
    a.chains = h->chains;
    a.X = h->L[0];
    a.Y = h->L[1];
    a.Z = h->L[2];
    a.N = h->N;
    return a;
}

extern "C" {

ising_status ising_mh_create(const ising_hmc_config *cfg, ising_mh_t **out) {
    g_mh_create_err[0] = 0;
    if (!cfg || !out) return mh_fail(nullptr, ISING_EINVAL, "null config or output pointer");
    *out = nullptr;
    if (cfg->kind != ISING_KIND_LATTICE)
        return mh_fail(nullptr, ISING_EINVAL, "Metropolis-Hastings runs on lattices only");
    if (cfg->dim < 1 || cfg->dim > 3) return mh_fail(nullptr, ISING_EINVAL, "dim must be 1..3");
    if (cfg->h) return mh_fail(nullptr, ISING_EINVAL, "per-site fields are not supported here");
    if (cfg->n_chains < 1 || cfg->n_chains > 65535)
        return mh_fail(nullptr, ISING_EINVAL, "n_chains must be 1..65535");
    int64_t N = 1;
    for (int d = 0; d < cfg->dim; ++d) {
        if (cfg->L[d] < 4 || cfg->L[d] % 2)
            return mh_fail(nullptr, ISING_EINVAL,
                           "extent L[%d]=%d: the checkerboard needs even extents >= 4", d, cfg->L[d]);
        N *= cfg->L[d];
    }
    if (N > ((int64_t)1 << 31)) return mh_fail(nullptr, ISING_EINVAL, "too many sites per chain");
    ising_mh *h = new (std::nothrow) ising_mh();
    if (!h) return mh_fail(nullptr, ISING_ENOMEM, "host allocation failed");
    auto bail = [&](ising_status st) {
        std::snprintf(g_mh_create_err, sizeof g_mh_create_err, "%s", h->err);
        mh_free(h);
        delete h;
        return st;
    };
    h->dim = cfg->dim;
    for (int d = 0; d < 3; ++d) h->L[d] = d < cfg->dim ? cfg->L[d] : 1;
    h->N = N;
    h->n_chains = cfg->n_chains;
    h->n_therm = cfg->n_therm;
    const int C = h->n_chains;
    h->packed = h->L[0] % 32 == 0;
    std::vector<MHChain> ch(C);
    std::vector<float> tab((size_t)C * 2 * MH_TAB, 0.0f);
    std::vector<uint32_t> ttab((size_t)C * 16, 0u);
    for (int c = 0; c < C; ++c) {
        const double beta = cfg->beta_chain ? cfg->beta_chain[c] : cfg->beta;
        const double h0 = cfg->h0_chain ? cfg->h0_chain[c] : cfg->h0;
        if (!(beta >= 0) || !std::isfinite(beta) || !std::isfinite(h0) || !std::isfinite(cfg->Jnn))
            return bail(mh_fail(h, ISING_EINVAL, "chain %d: need finite beta >= 0, J and h0", c));
        std::memset(&ch[c], 0, sizeof(MHChain));
        ch[c].beta = beta;
        ch[c].J = cfg->Jnn;
        ch[c].h = h0;
        for (int sp = 0; sp < 2; ++sp)
            for (int nb = -2 * h->dim; nb <= 2 * h->dim; ++nb) {
                const float pr = accept_prob(beta, cfg->Jnn, h0, sp ? 1 : -1, nb);
                tab[(size_t)c * 2 * MH_TAB + sp * MH_TAB + nb + 6] = pr;
                if ((nb + 2 * h->dim) % 2 == 0)   // cnt = number of +1 neighbours
                    ttab[(size_t)c * 16 + sp * 8 + (nb + 2 * h->dim) / 2] = accept_threshold(pr);
            }
    }
    if (cfg->stream) {
        h->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(mh_fail(h, ISING_ECUDA, "stream creation failed"));
        h->own_stream = true;
    }
    const size_t sb = h->packed ? (size_t)C * (N / 32) * 4 : (size_t)C * N;
    if ((h->packed ? cudaMalloc((void **)&h->sw, sb) : cudaMalloc((void **)&h->s, sb)) != cudaSuccess ||
        cudaMalloc((void **)&h->ttab, ttab.size() * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc((void **)&h->ptab, tab.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&h->acc, (size_t)C * 3 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void **)&h->chains, (size_t)C * sizeof(MHChain)) != cudaSuccess) {
        cudaGetLastError();
        return bail(mh_fail(h, ISING_ENOMEM, "device allocation failed (%zu bytes of spins)", sb));
    }
    // every spin +1: bytes of 1, or all bits set
    if (cudaMemsetAsync(h->packed ? (void *)h->sw : (void *)h->s, h->packed ? 0xff : 1, sb,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->ttab, ttab.data(), ttab.size() * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->acc, 0, (size_t)C * 3 * sizeof(unsigned long long), h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->ptab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->chains, ch.data(), (size_t)C * sizeof(MHChain), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return bail(mh_fail(h, ISING_ECUDA, "initialisation failed: %s",
                            cudaGetErrorString(cudaGetLastError())));
    *out = h;
    return ISING_OK;
}

ising_status ising_mh_sweeps(ising_mh_t *h, int64_t n, uint64_t seed) {
    if (!h) return ISING_EINVAL;
    nvtxRangePushA("ising_mh_sweeps");
    struct Pop { ~Pop() { nvtxRangePop(); } } pop;
    if (n < 0) return mh_fail(h, ISING_EINVAL, "n must be >= 0");
    if (h->sweep + n > (int64_t)0x7fffffff) return mh_fail(h, ISING_EINVAL, "sweep counter overflow");
    MHArgs a = mh_args(h);
    a.seed = seed;
    const int64_t groups = (h->N + 7) / 8;
    dim3 grid((unsigned)((groups + MH_THREADS - 1) / MH_THREADS), (unsigned)h->n_chains, 1);
    auto kern = h->dim == 3 ? mh_colour_kernel<3> : h->dim == 2 ? mh_colour_kernel<2> : mh_colour_kernel<1>;
    if (h->packed) {
        kern = h->dim == 3 ? mh_packed_kernel<3> : h->dim == 2 ? mh_packed_kernel<2> : mh_packed_kernel<1>;
        grid.x = (unsigned)((h->N / 32 + MH_THREADS - 1) / MH_THREADS);   // one word per thread
    } else if (h->L[0] % 8 == 0) {
        kern = h->dim == 3   ? mh_colour_row8_kernel<3>
               : h->dim == 2 ? mh_colour_row8_kernel<2>
                             : mh_colour_row8_kernel<1>;
        grid.x = (unsigned)((groups + 2 * MH_THREADS - 1) / (2 * MH_THREADS));   // two groups per thread
    }
    for (int64_t k = 0; k < n; ++k) {
        const int64_t sw = h->sweep + k;
        a.measure = sw >= h->n_therm;
        for (int c = 0; c < 2; ++c) {
            a.half = (uint32_t)(2 * sw + c);
            kern<<<grid, MH_THREADS, 0, h->stream>>>(a, c);
        }
        mh_measure_kernel<<<(h->n_chains + 127) / 128, 128, 0, h->stream>>>(a, h->n_chains);
        h->launches += 3;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return mh_fail(h, ISING_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
    }
    h->sweep += n;
    return ISING_OK;
}

ising_status ising_mh_sync(ising_mh_t *h) {
    if (!h) return ISING_EINVAL;
    const cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return mh_fail(h, ISING_ECUDA, "%s", cudaGetErrorString(e));
    return ISING_OK;
}

ising_status ising_mh_chain_sums(ising_mh_t *h, double *out) {
    if (!h || !out) return ISING_EINVAL;
    ising_status st = ising_mh_sync(h);
    if (st != ISING_OK) return st;
    std::vector<MHChain> ch(h->n_chains);
    if (cudaMemcpy(ch.data(), h->chains, sizeof(MHChain) * h->n_chains, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return mh_fail(h, ISING_ECUDA, "%s", cudaGetErrorString(cudaGetLastError()));
    for (int c = 0; c < h->n_chains; ++c)
        std::memcpy(out + (size_t)c * ISING_NSUMS, ch[c].sums, sizeof(double) * ISING_NSUMS);
    return ISING_OK;
}

ising_status ising_mh_observables(ising_mh_t *h, ising_obs *out) {
    if (!h || !out) return ISING_EINVAL;
    std::vector<double> sums((size_t)h->n_chains * ISING_NSUMS);
    ising_status st = ising_mh_chain_sums(h, sums.data());
    if (st != ISING_OK) return st;
    obs_from_sums(sums.data(), h->n_chains, h->sweep, out);
    return ISING_OK;
}

ising_status ising_mh_get_spins(ising_mh_t *h, int8_t *out) {
    if (!h || !out) return ISING_EINVAL;
    ising_status st = ising_mh_sync(h);
    if (st != ISING_OK) return st;
    if (h->packed) {
        const size_t nw = (size_t)h->n_chains * (h->N / 32);
        std::vector<uint32_t> w(nw);
        if (cudaMemcpy(w.data(), h->sw, nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return mh_fail(h, ISING_ECUDA, "%s", cudaGetErrorString(cudaGetLastError()));
        for (size_t k = 0; k < nw; ++k)
            for (int j = 0; j < 32; ++j) out[32 * k + j] = ((w[k] >> j) & 1u) ? 1 : -1;
        return ISING_OK;
    }
    if (cudaMemcpy(out, h->s, (size_t)h->n_chains * h->N, cudaMemcpyDeviceToHost) != cudaSuccess)
        return mh_fail(h, ISING_ECUDA, "%s", cudaGetErrorString(cudaGetLastError()));
    return ISING_OK;
}

ising_status ising_mh_set_spins(ising_mh_t *h, const int8_t *in, int64_t next_sweep) {
    if (!h || !in) return ISING_EINVAL;
    if (next_sweep < 0 || next_sweep > (int64_t)0x7fffffff)
        return mh_fail(h, ISING_EINVAL, "bad sweep index");
    const size_t n = (size_t)h->n_chains * h->N;
    for (size_t i = 0; i < n; ++i)
        if (in[i] != 1 && in[i] != -1) return mh_fail(h, ISING_EINVAL, "spin %zu is not +-1", i);
    ising_status st = ising_mh_sync(h);
    if (st != ISING_OK) return st;
    if (h->packed) {
        std::vector<uint32_t> w(n / 32, 0u);
        for (size_t i = 0; i < n; ++i)
            if (in[i] > 0) w[i / 32] |= 1u << (i % 32);
        if (cudaMemcpy(h->sw, w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return mh_fail(h, ISING_ECUDA, "%s", cudaGetErrorString(cudaGetLastError()));
    } else if (cudaMemcpy(h->s, in, n, cudaMemcpyHostToDevice) != cudaSuccess) {
        return mh_fail(h, ISING_ECUDA, "%s", cudaGetErrorString(cudaGetLastError()));
    }
    h->sweep = next_sweep;
    return ISING_OK;
}

int64_t ising_mh_sweep_index(const ising_mh_t *h) { return h ? h->sweep : -1; }
int64_t ising_mh_launch_count(const ising_mh_t *h) { return h ? h->launches : -1; }
const char *ising_mh_last_error(const ising_mh_t *h) { return h ? h->err : g_mh_create_err; }

void ising_mh_destroy(ising_mh_t *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    mh_free(h);
    delete h;
}

}  // extern "C"

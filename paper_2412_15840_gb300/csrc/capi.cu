// Host runtime and C ABI (include/sylv.h) of the N-dimensional Sylvester
// solver: plan construction (complex or real Schur factors, transform pass
// grouping, sweep tiling and schedules, workspace layout) and the
// stream-ordered launch sequences of Algorithm 3, of the mixed-precision
// refinement loop (FP64 or tensor-core residual), of Theorem 1 (sylv_evolve),
// of batched solves under one CUDA graph, and of the sweep autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "sylv_internal.h"

using cd = std::complex<double>;
using namespace sylv;

namespace {

struct Group {
    int first = 0, count = 0;
    int64_t L = 1, P = 1, R = 1;
    int Lt = 1, Rt = 1;
    int64_t tilesL = 1;
    size_t smem = 0;
    // tensor-core pass (one mode): operand geometry and the B images of
    // U^* (forward) and U (back) in the device pool
    int tc = 0;
    int mode1 = 0;                // first mode (L = 1): tiles of 64 columns
    int Kp = 0, Np = 0, lboA = 0, sboA = 0, sboB = 0, abytes = 0, bimg_bytes = 0;
    int tmem_cols = 0, nbuf = 1;
    const unsigned char *img[2] = {nullptr, nullptr};
    // real plan: the pass runs on the complex view of the real tensor (pairs of
    // entries adjacent in memory as one complex entry; L counts those pairs)
    int cview = 0;
    // FP64 residual group: three-multiplication products (re + im plane staged)
    int g3 = 0;
    // FP32 pass over one short mode, one thread per fibre (modeprod_fib.cu)
    int fib = 0;
};

// A mode after the first runs on the tensor cores when its fibres are at least
// 8 positions apart (tiles of 64 rows of the flattened (l, r) index stay
// mostly contiguous) and the operands fit in shared memory.
bool tc_mode_ok(int64_t L, int64_t n) {
    return L >= 8 && L < ((int64_t)1 << 30) && n >= 16 && n <= 80;
}
// The first mode (contiguous fibres) runs on the tensor cores with tiles of 64
// columns when it is not the last pass of a transform and n is a multiple of 8.
bool tc_mode1_ok(int64_t n, int64_t cols, int Nm) {
    return Nm >= 2 && n % 8 == 0 && n >= 16 && n <= 80 && cols >= 64;
}

void tc_geometry(Group &g, int n, bool mode1) {
    g.tc = 1;
    g.mode1 = mode1 ? 1 : 0;
    g.Kp = (n + 7) / 8 * 8;
    g.Np = (2 * n + 15) / 16 * 16;
    g.sboB = g.Kp * 32;
    if (mode1) {
        // 8-row groups adjacent, K-adjacent core matrices one padded column of
        // 16 groups apart: the staging stores (lanes along k) are conflict-free
        g.sboA = 128;
        g.lboA = 16 * 128 + 16;
        g.abytes = (g.Kp / 4) * g.lboA;
    } else {
        g.lboA = 128;
        g.sboA = g.Kp * 32 + 16;               // padding: conflict-free staging stores
        g.abytes = 16 * g.sboA;
    }
    g.bimg_bytes = (g.Np / 8) * g.sboB;
    int need = std::max(g.Np, n + 16 * ((n + 15) / 16));
    int cols = 32;
    while (cols < need) cols *= 2;
    g.tmem_cols = cols;
    // two A buffers and accumulators (MMAs of the next tile overlap the
    // current tile's epilogue) when they fit next to the B images
    const size_t one = (size_t)2 * g.abytes;
    const size_t slack = mode1 ? 4096 : 0;     // keeps the padded A images inside the allocation
    g.nbuf = (size_t)2 * g.bimg_bytes + 2 * one + slack <= (size_t)TC_SMEM_MAX ? 2 : 1;
    g.smem = (size_t)2 * g.bimg_bytes + (size_t)g.nbuf * one + slack;
}

struct TimedPhase {
    int phase;
    cudaEvent_t a, b;
    int launches;
};

// One sweep configuration: kernel arguments (tables in `dbuf`), launch shape.
struct SweepConfig {
    SweepArgs a{};
    int threads = 256, grid = 1, per_sm = 1;
    size_t smem = 0;
    void *dbuf = nullptr;
    // device copy of `a` with the plan's factor pointers filled in (Y, cnt and
    // flags are per call): the batched sweep reads each equation's from here
    const SweepArgs *dargs = nullptr;
};

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

std::mutex g_init_mu;
std::set<int> g_init_devices;

sylv_status ensure_init(int dev) {
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (g_init_devices.count(dev)) return SYLV_OK;
    if (kernels_init(dev) != cudaSuccess) return SYLV_ERR_CUDA;
    g_init_devices.insert(dev);
    return SYLV_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct sylv_plan_s {
    int device = 0;
    int prec = SYLV_FP64;
    double rtol = 1e-10;
    int max_refine = 5;
    int N_in = 0;
    std::vector<int64_t> n_in;
    int64_t nrhs = 1;
    int Nm = 0;
    int64_t n[MAXM] = {};
    int64_t S[MAXM] = {};
    int orig[MAXM] = {};
    int64_t ntot = 1;
    cd sigma = 0.0;
    std::vector<std::vector<cd>> Ah, Qh, Th;   // per input mode

    void *dpool = nullptr;
    const void *Uh64[MAXM] = {}, *U64[MAXM] = {}, *A64[MAXM] = {}, *T64[MAXM] = {};
    const void *Uh32[MAXM] = {}, *U32[MAXM] = {}, *T32[MAXM] = {};
    const double *d64[MAXM] = {};

    std::vector<Group> tgroups;   // transform passes in the working precision
    std::vector<Group> rgroups;   // FP64 residual passes
    // SYLV_MIXED_FP32_EMU: residual passes on the bf16 tensor cores (one per mode)
    struct OzPass {
        int j = 0, mode1 = 0, n = 0, Kp = 0, Np = 0, lboX = 0, sboX = 0, sboAd = 0;
        int ximg_bytes = 0, aimg_bytes = 0, tmem_cols = 0, eA = 0, rstage_off = 0;
        int64_t L = 1, R = 1, tilesL = 1;
        size_t smem = 0;
        const unsigned char *aimg = nullptr;   // digits of A_j (A_1 + sigma I)
        const unsigned char *eimg = nullptr;   // digits of exp(t A_j) (sylv_evolve)
        int eE = 0;                            // their scale exponent
    };
    std::vector<unsigned char> Eimg_host;      // staging of the exp(t A_j) digits
    std::vector<OzPass> ozpasses;
    bool oz = false;              // every mode qualifies: the residual runs on the tensor cores
    bool tc_plain = false;        // tensor-core passes without the TMA-fed pipeline
    int tgroup_max = 0;           // fusion width of the CUDA-core transform groups (0: automatic)

    SweepConfig sweep;            // Y, T, diag, flags, counters filled per launch
    int64_t cnt_capacity = 0;     // tile counters the workspace holds (any tuned tiling)
    double den_scale = 1.0;       // power of two for the sweep's reciprocals
    void *inv_tab = nullptr;      // reciprocal per multi-index (when within INV_TABLE_MAX)
    int num_sms = 1;
    long long timeout_cycles = 4000000000LL;   // per dependency wait
    int fault_tile = -1;                       // test hook (sylv_tuning.fault_tile - 1)

    // Theorem 1 (sylv_evolve): FP64 composition passes with exp(t A_j), the
    // negated A_j for the first step of Eq. (C), and the last t prepared
    std::vector<Group> egroups;
    const void *nA64[MAXM] = {}, *E64[MAXM] = {};
    std::vector<double> Ehost;
    double evolve_t = 0.0;
    bool evolve_ready = false;
    cd evolve_eps = 1.0;          // exp(t * sigma): the singleton modes' exponentials

    // Remark 1: every T_j diagonal to rounding -> entrywise-division sweep
    bool diag_sweep = false;
    DiagArgs diag{};

    double min_den = 0.0, max_den = 0.0;
    size_t off_cnt = 0, off_W = 0, off_R = 0, ws_bytes = 0;

    bool timing = false;
    std::vector<TimedPhase> tphases;
    std::vector<cudaEvent_t> ev_free;
    int64_t timed_solves = 0;
    int last_launches = 0;

    ~sylv_plan_s() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != device) cudaSetDevice(device);
        for (auto &p : tphases) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto e : ev_free) cudaEventDestroy(e);
        if (dpool) cudaFree(dpool);
        if (sweep.dbuf) cudaFree(sweep.dbuf);
        if (inv_tab) cudaFree(inv_tab);
        if (cur >= 0 && cur != device) cudaSetDevice(cur);
    }

    // real-arithmetic variant (sylv_plan_create_real): real Schur factors per
    // input mode, the pair rotations V_j (4 complex entries per index pair), the
    // real quasi-triangular T_j and the V_j on the device; Th holds the complex
    // triangular T~_j = V_j^* T_j V_j, Qh the real Q_j
    bool real = false;
    std::vector<std::vector<double>> Qr, Tr;
    std::vector<std::vector<cd>> Vh;
    bool has_pairs[MAXM] = {};
    const void *Tr64[MAXM] = {}, *Tr32[MAXM] = {}, *V64[MAXM] = {}, *V32[MAXM] = {};

    bool fp64() const { return prec == SYLV_FP64; }
    bool emu() const { return prec == SYLV_MIXED_FP32_EMU; }
    // element kinds and sizes of the FP64 tensors (B, X, R) and the FP32 working tensor
    int khi() const { return real ? ELEM_R64 : ELEM_C128; }
    int klo() const { return real ? ELEM_R32 : ELEM_C64; }
    size_t ehi() const { return real ? 8 : 16; }
    size_t elo() const { return real ? 4 : 8; }
};

namespace {

// ----------------------------------------------------------------- tiling --

bool choose_tile(int64_t L, int64_t P, int64_t R, int64_t Et, int64_t Eh, int &Lt, int &Rt) {
    int64_t lt, rt;
    if (L * P <= Et) {
        lt = L;
        rt = std::max<int64_t>(1, std::min<int64_t>(R, Et / (L * P)));
    } else if (L < 32) {
        lt = L;
        rt = 1;
    } else {
        lt = (Et / P) / 32 * 32;
        if (lt < 32) lt = 32;
        if (lt * P > Eh) lt = std::max<int64_t>(1, Eh / P);
        lt = std::min<int64_t>(lt, L);
        rt = 1;
    }
    if (lt * P * rt > Eh) return false;
    Lt = (int)lt;
    Rt = (int)rt;
    return true;
}

// [Re M^T | Im M^T] of an n x n complex matrix as 6 base-256 digits of |m| / 2^e
// (bf16, the B-operand layout of the digit-product pass); returns e, with
// |entries| < 2^(e - 1).
template <typename Pass>
int digit_images(const std::vector<std::complex<double>> &M, const Pass &o, unsigned char *img) {
    const int n = o.n;
    double amax = 0.0;
    for (auto &z : M) amax = std::max(amax, std::max(std::fabs(z.real()), std::fabs(z.imag())));
    const int e = amax > 0.0 ? std::ilogb(amax) + 2 : 0;
    std::memset(img, 0, (size_t)6 * o.aimg_bytes);
    for (int ii = 0; ii < 2 * n; ++ii)
        for (int k = 0; k < n; ++k) {
            const int i = ii < n ? ii : ii - n;
            const std::complex<double> z = M[(size_t)(i + k * n)];
            const double v = ii < n ? z.real() : z.imag();
            const uint64_t F = (uint64_t)std::floor(std::ldexp(std::fabs(v), 48 - e));
            const size_t off = (size_t)(ii / 8) * o.sboAd + (size_t)(k / 8) * 128 +
                               (size_t)(ii % 8) * 16 + (size_t)(k % 8) * 2;
            for (int u = 0; u < 6; ++u) {
                const uint32_t d = (uint32_t)(F >> (40 - 8 * u)) & 0xFFu;
                const float fd = (float)d;
                uint32_t fb;
                std::memcpy(&fb, &fd, 4);
                uint16_t b = (uint16_t)(fb >> 16);        // exact: d has <= 8 bits
                if (d && v < 0) b |= 0x8000u;
                std::memcpy(img + (size_t)u * o.aimg_bytes + off, &b, 2);
            }
        }
    return e;
}

// Residual passes on the tensor cores: every non-singleton mode needs
// 8 <= n <= 64, and fibres at least 8 apart for a later mode (tiles of 64 rows of
// the flattened (l, r) index), or at least 64 columns for the first mode.
// Returns false when some mode does not qualify.
bool make_oz_passes(const sylv_plan_s &p, std::vector<sylv_plan_s::OzPass> &out) {
    out.clear();
    if (p.Nm == 0) return false;
    const int64_t tot = p.ntot * p.nrhs;
    for (int j = 0; j < p.Nm; ++j) {
        const int64_t n = p.n[j], L = p.S[j];
        if (n < 8 || n > 64) return false;
        sylv_plan_s::OzPass o;
        o.j = j;
        o.n = (int)n;
        o.mode1 = j == 0 ? 1 : 0;
        o.L = L;
        o.R = tot / (L * n);
        if (o.mode1) {
            if (o.R < 64) return false;
        } else if (L < 8 || L >= ((int64_t)1 << 30)) {
            return false;
        }
        o.tilesL = 1;
        o.Kp = (int)((n + 15) / 16 * 16);
        o.Np = (int)((2 * n + 15) / 16 * 16);
        if (o.mode1) {              // lanes along k: K-adjacent core matrices one padded column apart
            o.sboX = 128;
            o.lboX = 16 * 128 + 16;
            o.ximg_bytes = (o.Kp / 8) * o.lboX;
        } else {                    // lanes along l: padded 8-row groups
            o.lboX = 128;
            o.sboX = (o.Kp / 8) * 128 + 16;
            o.ximg_bytes = 16 * o.sboX;
        }
        o.sboAd = (o.Kp / 8) * 128;
        o.aimg_bytes = (o.Np / 8) * o.sboAd;
        int cols = 32;
        while (cols < 4 * o.Np) cols *= 2;
        o.tmem_cols = cols;
        // epilogue operand slots (4 per 32 columns, 16 B per thread and slot):
        // appended after the digit images where they fit (the K padding of the
        // X images, zeroed once, then stays zero), else in the X digit images,
        // free while the epilogue runs (the padding is zeroed again per tile)
        const size_t rstage = (size_t)4 * ((n + 31) / 32) * 512 * 16;
        const size_t xarea = (size_t)6 * o.ximg_bytes;
        o.rstage_off = 6 * o.aimg_bytes;
        o.smem = (size_t)6 * o.aimg_bytes + xarea + 4096;
        if (rstage > xarea || o.smem + rstage <= (size_t)TC_SMEM_MAX) {
            o.rstage_off = (int)(o.smem);
            o.smem += rstage;
        }
        if (o.smem > (size_t)TC_SMEM_MAX) return false;
        out.push_back(o);
    }
    return true;
}

sylv_status make_groups(const sylv_plan_s &p, bool fp64, bool composition, int group_max,
                        bool allow_tc,
                        std::vector<Group> &out) {
    const int64_t esz = (fp64 ? 16 : 8) / (p.real ? 2 : 1);
    const bool plane = !composition && fp64 && !p.real;   // residual's re + im plane
    const int64_t Et = fp64 ? 2048 : 4096;
    const int64_t Eh = fp64 ? 8192 : 16384;
    out.clear();
    const int64_t tot = p.ntot * p.nrhs;
    if (p.Nm == 0) {
        Group g;
        g.first = 0; g.count = 0; g.L = 1; g.P = 1; g.R = tot;
        choose_tile(1, 1, tot, Et, Eh, g.Lt, g.Rt);
        g.tilesL = 1;
        g.smem = (size_t)(g.Lt * g.Rt) * esz;
        out.push_back(g);
        return SYLV_OK;
    }
    const bool use_tc = composition && !fp64 && allow_tc;
    // A real plan's mode with an even stride runs on the tensor cores over the
    // complex view of the float32 tensor: two entries adjacent in memory differ
    // in an earlier mode's index, so a later mode's product treats them alike,
    // and the real Q_j (a complex matrix with zero imaginary part) maps the pair
    // (x_2a, x_2a+1) as one complex entry x_2a + i x_2a+1.
    auto tc_ok = [&](int jj) {
        if (!use_tc) return false;
        if (!p.real) return tc_mode_ok(p.S[jj], p.n[jj]);
        return p.S[jj] % 2 == 0 && tc_mode_ok(p.S[jj] / 2, p.n[jj]);
    };
    // one-thread-per-fibre FP32 pass: complex modes with n <= FIB_NMAX outside
    // the TMA-fed tensor-core pass (fibres 64-aligned along l), and not fused
    // with a neighbour (checked below)
    const bool use_fib = composition && !fp64 && !p.real;
    auto tma_ok = [&](int jj) {
        return tc_ok(jj) && jj > 0 && p.S[jj] % 64 == 0 && p.n[jj] <= 64;
    };
    auto fib_ok = [&](int jj) {
        return use_fib && p.n[jj] >= 2 && p.n[jj] <= FIB_NMAX && !tma_ok(jj);
    };
    int j = 0;
    while (j < p.Nm) {
        Group g;
        g.first = j;
        g.L = p.S[j];
        if (fib_ok(j) && p.n[j] >= 16) {
            g.count = 1;
            g.P = p.n[j];
            g.R = tot / (g.L * g.P);
            g.fib = 1;
            g.smem = (size_t)p.n[j] * fib_nx((int)p.n[j]) * 8;
            out.push_back(g);
            j += 1;
            continue;
        }
        const bool m1 = use_tc && !p.real && j == 0 && tc_mode1_ok(p.n[0], tot / p.n[0], p.Nm);
        if (m1 || tc_ok(j)) {
            g.count = 1;
            g.P = p.n[j];
            g.R = tot / (g.L * g.P);
            if (p.real) {
                g.cview = 1;
                g.L = p.S[j] / 2;
            }
            g.tilesL = m1 ? 1 : (g.L + 63) / 64;
            tc_geometry(g, (int)p.n[j], m1);
            out.push_back(g);
            j += 1;
            continue;
        }
        int64_t Pcap = Et / std::min<int64_t>(g.L, 32);
        if (group_max > 0) Pcap = std::min<int64_t>(Pcap, group_max);
        g.P = p.n[j];
        g.count = 1;
        while (j + g.count < p.Nm && g.count < MAXG && g.P * p.n[j + g.count] <= Pcap &&
               p.S[j + g.count] == g.L * g.P && !tc_ok(j + g.count))
            g.P *= p.n[j + g.count], g.count++;
        g.R = tot / (g.L * g.P);
        if (g.count == 1 && fib_ok(j)) {      // not fused: one thread per fibre
            g.fib = 1;
            g.smem = (size_t)p.n[j] * fib_nx((int)p.n[j]) * 8;
            out.push_back(g);
            j += 1;
            continue;
        }
        if (!choose_tile(g.L, g.P, g.R, Et, Eh, g.Lt, g.Rt)) return SYLV_ERR_SHAPE;
        g.tilesL = (g.L + g.Lt - 1) / g.Lt;
        int64_t E = (int64_t)g.Lt * g.P * g.Rt;
        g.g3 = plane ? 1 : 0;
        // composition: two tiles (ping-pong); residual: the tile and its
        // re + im plane (FP64 only); otherwise one tile
        g.smem = (size_t)(E * esz * ((composition && g.count > 1) ? 2 : 1));
        if (g.g3) g.smem += (size_t)E * 8;
        if (g.smem > 200 * 1024) return SYLV_ERR_SHAPE;
        out.push_back(g);
        j += g.count;
    }
    return SYLV_OK;
}

// Sweep tile extents: balanced doubling of the block with the most blocks
// left until a tile holds `target` entries (or the explicit tuning blocks).
void choose_blocks(const sylv_plan_s &p, int target, const sylv_tuning *tu, int *b) {
    bool manual = false;
    for (int j = 0; j < p.Nm; ++j) {
        b[j] = 1;
        if (tu && p.orig[j] < 64 && tu->block[p.orig[j]] > 0) {
            b[j] = (int)std::min<int64_t>(tu->block[p.orig[j]], p.n[j]);
            manual = true;
        }
    }
    // real variant: a mode with 2 x 2 blocks needs an even extent (or the whole
    // mode) so that no tile splits a block
    for (int j = 0; j < p.Nm; ++j)
        if (p.real && p.has_pairs[j] && b[j] < p.n[j] && (b[j] & 1))
            b[j] = (int)std::min<int64_t>(b[j] + 1, p.n[j]);
    if (manual) return;
    for (;;) {
        int best = -1;
        double bestr = 1.0;
        int64_t prod = 1;
        for (int j = 0; j < p.Nm; ++j) prod *= b[j];
        for (int j = 0; j < p.Nm; ++j) {
            if (b[j] >= p.n[j] || b[j] >= SWEEP_BMAX) continue;
            int64_t nb = std::min<int64_t>(std::min<int64_t>(2 * b[j], p.n[j]), SWEEP_BMAX);
            if (prod / b[j] * nb > target) continue;
            double r = (double)p.n[j] / b[j];
            if (r > bestr) { bestr = r; best = j; }
        }
        if (best < 0) break;
        b[best] = (int)std::min<int64_t>(2 * b[best], p.n[best]);
    }
}

int64_t tiles_for(const sylv_plan_s &p, const int *b) {
    int64_t ts = 1;
    for (int j = 0; j < p.Nm; ++j) ts *= (p.n[j] + b[j] - 1) / b[j];
    return ts * p.nrhs;
}

// The plan's factor pointers of the sweep in its working precision.
void fill_sweep_ptrs(const sylv_plan_s &p, SweepArgs &a, bool fp64) {
    for (int j = 0; j < p.Nm; ++j) {
        a.T[j] = fp64 ? p.T64[j] : p.T32[j];
        a.d[j] = p.d64[j];
        a.Tr[j] = fp64 ? p.Tr64[j] : p.Tr32[j];
        a.Vp[j] = p.has_pairs[j] ? (fp64 ? p.V64[j] : p.V32[j]) : nullptr;
    }
    a.den_scale = p.den_scale;
    a.inv_tab = p.inv_tab;
}

// Host tables of one sweep configuration (tile extents b, `threads` per CTA),
// uploaded into a device buffer of its own, followed by a device copy of the
// configuration's arguments.
sylv_status build_sweep(const sylv_plan_s &p, const int *b, int threads, SweepConfig &cfg,
                        int ctas_per_sm = 0, int sub = 0) {
    SweepArgs &a = cfg.a;
    a = SweepArgs{};
    a.Nm = p.Nm;
    int64_t ts = 1;
    a.nin = 0;
    int bs = 1;
    a.Lin = 1;
    for (int j = 0; j < p.Nm; ++j) {
        a.n[j] = p.n[j];
        a.S[j] = p.S[j];
        a.b[j] = b[j];
        a.qpos[j] = b[j] > 1 ? a.nin : -1;
        a.Bc[j] = (int)((p.n[j] + b[j] - 1) / b[j]);
        a.TS[j] = ts;
        ts *= a.Bc[j];
        if (b[j] > 1) {
            a.inmode[a.nin] = j;
            a.BS[a.nin] = bs;
            bs *= b[j];
            a.nin++;
            a.Lin += b[j] - 1;
        }
    }
    a.Pt = bs;
    if (a.Pt > 8192) return SYLV_ERR_SHAPE;
    a.ntiles1 = ts;
    a.ntot = p.ntot;
    if (ts > 0x7fffffffLL || ts * p.nrhs > 0x7fffffffLL) return SYLV_ERR_SHAPE;
    a.ntiles = ts * p.nrhs;
    a.sig_re = p.sigma.real();
    a.sig_im = p.sigma.imag();
    a.timeout_cycles = p.timeout_cycles;
    a.fault_tile = p.fault_tile;
    a.real = p.real ? 1 : 0;

    // in-tile schedule: box offsets sorted by their distance from the tile end
    std::vector<int> lvl(a.Pt), cntl(a.Lin + 1, 0);
    for (int e = 0; e < a.Pt; ++e) {
        int sum = 0;
        for (int q = 0; q < a.nin; ++q) sum += (e / a.BS[q]) % a.b[a.inmode[q]];
        lvl[e] = sum;
        cntl[sum + 1]++;
    }
    std::vector<int> lev(a.Lin + 1, 0), sched(a.Pt, 0);
    for (int l = 0; l < a.Lin; ++l) lev[l + 1] = lev[l] + cntl[l + 1];
    {
        std::vector<int> pos(lev.begin(), lev.end() - 1);
        for (int e = 0; e < a.Pt; ++e) sched[pos[lvl[e]]++] = e;
    }
    // for full tiles: the schedule as box offsets, and every box offset's
    // in-tile coordinates packed into 64 bits, ceil(log2 b) bits per mode
    a.bmax = 1;
    int cbits = 0;
    for (int q = 0; q < a.nin; ++q) {
        const int bq = a.b[a.inmode[q]];
        a.bmax = std::max(a.bmax, bq);
        int w = 1;
        while ((1 << w) < bq) ++w;
        a.cshift[q] = cbits;
        a.cmask[q] = (1u << w) - 1u;
        cbits += w;
    }
    a.fast = cbits <= 64 ? 1 : 0;
    std::vector<int> sched_e(a.Pt, 0);
    std::vector<unsigned long long> coord(a.Pt, 0ull);
    for (int qq = 0; qq < a.Pt; ++qq) {
        int e = 0;
        for (int q = 0; q < a.nin; ++q) {
            const int bq = a.b[a.inmode[q]];
            const int apq = (sched[qq] / a.BS[q]) % bq;
            e += (bq - 1 - apq) * a.BS[q];
        }
        sched_e[qq] = e;
    }
    // element offsets of the box positions from the tile's first entry (32-bit
    // when the tensor per right-hand side is below 2^31 entries)
    a.use_offs = a.fast && p.ntot < ((int64_t)1 << 31) ? 1 : 0;
    std::vector<int> offs(a.use_offs ? a.Pt : 0, 0);
    if (a.fast)
        for (int e = 0; e < a.Pt; ++e) {
            unsigned long long c = 0;
            int64_t off = 0;
            for (int q = 0; q < a.nin; ++q) {
                const int t = (e / a.BS[q]) % a.b[a.inmode[q]];
                c |= (unsigned long long)t << a.cshift[q];
                off += (int64_t)t * a.S[a.inmode[q]];
            }
            coord[e] = c;
            if (a.use_offs) offs[(size_t)e] = (int)off;
        }

    // tile order: by level sum_j (Bc_j - 1 - I_j), then right-hand side, then id
    int maxlev = 0;
    for (int j = 0; j < p.Nm; ++j) maxlev += a.Bc[j] - 1;
    std::vector<int> tl((size_t)ts);
    std::vector<int64_t> cnt((size_t)maxlev + 2, 0);
    for (int64_t t = 0; t < ts; ++t) {
        int sum = 0;
        for (int j = 0; j < p.Nm; ++j) sum += a.Bc[j] - 1 - (int)((t / a.TS[j]) % a.Bc[j]);
        tl[(size_t)t] = sum;
        cnt[(size_t)sum + 1]++;
    }
    for (int l = 0; l <= maxlev; ++l) cnt[(size_t)l + 1] += cnt[(size_t)l];
    std::vector<int> by_level((size_t)ts);
    {
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t t = 0; t < ts; ++t) by_level[(size_t)pos[(size_t)tl[(size_t)t]]++] = (int)t;
    }
    std::vector<int> order((size_t)(ts * p.nrhs));
    size_t w = 0;
    for (int l = 0; l <= maxlev; ++l)
        for (int64_t r = 0; r < p.nrhs; ++r)
            for (int64_t q = cnt[(size_t)l]; q < cnt[(size_t)l + 1]; ++q)
                order[w++] = (int)(r * ts + by_level[(size_t)q]);

    // FP64 reciprocals, tile values, one staged block of T, diagonal T blocks
    const size_t esz = p.fp64() ? 16 : 8;
    int td = 0;
    for (int q = 0; q < a.nin; ++q) {
        a.tdoff[q] = td;
        td += a.b[a.inmode[q]] * a.b[a.inmode[q]];
    }
    a.tdsize = td;
    cfg.threads = threads;
    cfg.smem = (size_t)a.Pt * (esz + 16) + ((size_t)SWEEP_KCH * a.bmax + td) * esz +
               (a.fast ? (size_t)a.Pt * 12 : 0) +    // packed coordinates + schedule
               (a.use_offs ? (size_t)a.Pt * 4 : 0);  // box offsets
    if (cfg.smem > 200 * 1024) return SYLV_ERR_SHAPE;
    // FP64 complex strips by three multiplications need the re + im plane of the
    // staged T block; it is reserved only where it costs no resident CTA, in the
    // single-equation sweep and in the batched one (measured: a plane that took
    // one CTA per SM slowed the 512-equation batch by 5%)
    a.g3 = 0;
    if (p.fp64() && !p.real) {
        const size_t plane = (size_t)SWEEP_KCH * a.bmax * 8 + 8;
        const int cap = ctas_per_sm > 0 ? ctas_per_sm : 1 << 20;
        const int s0 = std::min(cap, sweep_blocks_per_sm(1, threads, cfg.smem, 0));
        const int s1 = std::min(cap, sweep_blocks_per_sm(1, threads, cfg.smem + plane, 0));
        const int b0 = sweep_batch_blocks_per_sm(1, threads, cfg.smem, 0);
        const int b1 = sweep_batch_blocks_per_sm(1, threads, cfg.smem + plane, 0);
        if (s1 >= s0 && s1 >= 1 && b1 >= b0 && cfg.smem + plane <= 200 * 1024) {
            a.g3 = 1;
            cfg.smem += plane;
        }
    }

    // device tables: order | sched | lev | sched_e | coord | offs
    size_t o_order = 0;
    size_t o_sched = align256(o_order + order.size() * 4);
    size_t o_lev = align256(o_sched + sched.size() * 4);
    size_t o_se = align256(o_lev + lev.size() * 4);
    size_t o_coord = align256(o_se + sched_e.size() * 4);
    size_t o_offs = align256(o_coord + coord.size() * 8);
    size_t o_args = align256(o_offs + offs.size() * 4);
    size_t total = align256(o_args + sizeof(SweepArgs));
    std::vector<unsigned char> host(total, 0);
    std::memcpy(host.data() + o_order, order.data(), order.size() * 4);
    std::memcpy(host.data() + o_sched, sched.data(), sched.size() * 4);
    std::memcpy(host.data() + o_lev, lev.data(), lev.size() * 4);
    std::memcpy(host.data() + o_se, sched_e.data(), sched_e.size() * 4);
    std::memcpy(host.data() + o_coord, coord.data(), coord.size() * 8);
    if (!offs.empty()) std::memcpy(host.data() + o_offs, offs.data(), offs.size() * 4);
    if (cudaMalloc(&cfg.dbuf, total) != cudaSuccess) {
        cudaGetLastError();
        cfg.dbuf = nullptr;
        return SYLV_ERR_OOM;
    }
    if (cudaMemcpy(cfg.dbuf, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess)
        return SYLV_ERR_CUDA;
    unsigned char *base = (unsigned char *)cfg.dbuf;
    a.order = (const int *)(base + o_order);
    a.sched = (const int *)(base + o_sched);
    a.lev_start = (const int *)(base + o_lev);
    a.sched_e = (const int *)(base + o_se);
    a.coord = (const unsigned long long *)(base + o_coord);
    a.offs = (const int *)(base + o_offs);
    cfg.dargs = (const SweepArgs *)(base + o_args);

    // persistent grid: every SM holds as many tiles as fit, or the requested
    // number (fewer CTAs per SM shorten each tile's latency on the dependency
    // chain at the cost of tiles in flight)
    int per = sweep_blocks_per_sm(p.fp64(), cfg.threads, cfg.smem, a.real);
    if (per < 1) per = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per) per = ctas_per_sm;
    cfg.per_sm = per;
    cfg.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)p.num_sms * per, a.ntiles));
    // far strips ahead of the full dependency wait pay where the sweep is bound by
    // its dependency chain: at most two tiles per level for each resident CTA
    a.far_split = a.ntiles <= (int64_t)2 * cfg.grid * (maxlev + 1) ? 1 : 0;
    // lanes per entry in the in-tile wavefront: 4 on the latency-bound FP32 path,
    // else 1 (the FP64 path is bound by its pipe; a throughput-bound sweep by
    // issue slots)
    a.sub = sub > 0 ? sub : (!p.fp64() && a.far_split ? 4 : 1);
    SweepArgs full = a;
    fill_sweep_ptrs(p, full, p.fp64());
    if (cudaMemcpy(base + o_args, &full, sizeof(full), cudaMemcpyHostToDevice) != cudaSuccess)
        return SYLV_ERR_CUDA;
    return SYLV_OK;
}

// ------------------------------------------------------------- launchers --

struct Ctx {
    sylv_plan_s *p;
    cudaStream_t st;
    DevFlags *flags;
    int *cnt;
    int launches = 0;
    int phase_launches = 0;
    int cur_phase = -1;
    cudaEvent_t cur_ev = nullptr;
};

cudaEvent_t take_event(sylv_plan_s *p) {
    if (!p->ev_free.empty()) {
        cudaEvent_t e = p->ev_free.back();
        p->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void phase_begin(Ctx &c, int ph) {
    c.cur_phase = ph;
    c.phase_launches = 0;
    if (!c.p->timing) return;
    c.cur_ev = take_event(c.p);
    cudaEventRecord(c.cur_ev, c.st);
}

void phase_end(Ctx &c) {
    if (c.p->timing && c.cur_ev) {
        cudaEvent_t b = take_event(c.p);
        cudaEventRecord(b, c.st);
        c.p->tphases.push_back({c.cur_phase, c.cur_ev, b, c.phase_launches});
        c.cur_ev = nullptr;
    }
    c.cur_phase = -1;
}

void count(Ctx &c) { c.launches++; c.phase_launches++; }

cudaError_t run_groups(Ctx &c, const std::vector<Group> &gs, bool fp64, int which,
                       const void *first_in, int first_in_kind, void *work, int work_kind,
                       void *last_out, int last_out_kind, int last_epi, const int *done,
                       const void *const *mats = nullptr, const void *aux = nullptr,
                       cd scale = 1.0) {
    // which: 0 forward (U^*), 1 back (U); `mats` replaces both (per mode)
    sylv_plan_s *p = c.p;
    for (size_t gi = 0; gi < gs.size(); ++gi) {
        const Group &g = gs[gi];
        MPArgs a{};
        a.G = g.count;
        for (int m = 0; m < g.count; ++m) {
            int j = g.first + m;
            a.gn[m] = (int)p->n[j];
            if (mats) a.mats[m] = mats[j];
            else if (fp64) a.mats[m] = which == 0 ? p->Uh64[j] : p->U64[j];
            else a.mats[m] = which == 0 ? p->Uh32[j] : p->U32[j];
        }
        a.B = aux;
        a.sig_re = scale.real();
        a.sig_im = scale.imag();
        a.L = g.L; a.P = g.P; a.R = g.R; a.Lt = g.Lt; a.Rt = g.Rt; a.tilesL = g.tilesL;
        a.flags = c.flags;
        a.done = done;
        const bool first = gi == 0, last = gi + 1 == gs.size();
        a.in = first ? first_in : work;
        int in_kind = first ? first_in_kind : work_kind;
        a.out = last ? last_out : work;
        int out_kind = last ? last_out_kind : work_kind;
        int epi = last ? last_epi : EPI_STORE;
        if (g.count == 0 && a.in == a.out && epi == EPI_STORE) continue;   // identity
        if (g.fib) {
            cudaError_t e = launch_modeprod_fib(in_kind, out_kind, epi, a, p->num_sms, c.st);
            if (e != cudaSuccess) return e;
            count(c);
            continue;
        }
        if (g.tc) {
            if (g.cview) {     // float32 / float64 tensors as complex64 / complex128 pairs
                if (in_kind == ELEM_R32) in_kind = ELEM_C64;
                if (out_kind == ELEM_R32) out_kind = ELEM_C64;
                if (out_kind == ELEM_R64) out_kind = ELEM_C128;
            }
            if (in_kind != ELEM_C64 && !(g.mode1 && in_kind == ELEM_C128))
                return cudaErrorInvalidValue;
            if (mats) return cudaErrorInvalidValue;   // B images hold U^* and U only
            TCArgs t{};
            t.in = a.in;
            t.out = a.out;
            t.bimg = g.img[which];
            t.n = (int)g.P;
            t.mode1 = g.mode1;
            t.in_c128 = in_kind == ELEM_C128 ? 1 : 0;
            t.Kp = g.Kp; t.Np = g.Np; t.lboA = g.lboA; t.sboA = g.sboA; t.sboB = g.sboB;
            t.abytes = g.abytes;
            t.bimg_bytes = g.bimg_bytes;
            t.tmem_cols = g.tmem_cols;
            t.nbuf = g.nbuf;
            t.L = g.L; t.R = g.R; t.tilesL = g.tilesL;
            t.flags = c.flags;
            t.done = done;
            // TMA-fed warp-specialised pass where it applies, else the register-staged one
            cudaError_t e = p->tc_plain ? cudaErrorNotSupported
                                        : launch_modeprod_tcw(epi, t, p->num_sms, c.st);
            if (e == cudaSuccess) {
                count(c);
                continue;
            }
            if (e != cudaErrorNotSupported) return e;
            const int64_t tiles = g.mode1 ? (g.R + 63) / 64 : (g.L * g.R + 63) / 64;
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, p->num_sms));
            e = launch_modeprod_tc(epi, t, grid, g.smem, c.st);
            if (e != cudaSuccess) return e;
            count(c);
            continue;
        }
        cudaError_t e = launch_modeprod(fp64, in_kind, out_kind, epi, a, g.smem, c.st);
        if (e != cudaSuccess) return e;
        count(c);
    }
    return cudaSuccess;
}

// R = B - sigma X - sum_j M_j (x)_j X over the FP64 residual passes, M_j = A_j
// (or the given per-mode matrices, with the given sigma; each matrix carries the
// plane re + im after its entries)
cudaError_t run_residual(Ctx &c, const void *B, const void *X, void *R, const int *done,
                         const void *const *mats = nullptr, const cd *sig = nullptr) {
    sylv_plan_s *p = c.p;
    const cd sg = sig ? *sig : p->sigma;
    for (size_t gi = 0; gi < p->rgroups.size(); ++gi) {
        const Group &g = p->rgroups[gi];
        MPArgs a{};
        a.G = g.count;
        for (int m = 0; m < g.count; ++m) {
            int j = g.first + m;
            a.gn[m] = (int)p->n[j];
            a.mats[m] = mats ? mats[j] : p->A64[j];
        }
        a.L = g.L; a.P = g.P; a.R = g.R; a.Lt = g.Lt; a.Rt = g.Rt; a.tilesL = g.tilesL;
        a.in = X;
        a.out = R;
        a.B = B;
        a.sig_re = sg.real();
        a.sig_im = sg.imag();
        a.first = gi == 0;
        a.g3 = g.g3;
        // four rows per thread save loads where the pass fills the GPU several
        // times; a smaller pass keeps one row per thread and four times the
        // threads (measured: 64^4 residual 22.3 -> 21.8 ms, 33 x 45 x 71 0.27 ->
        // 0.31 ms with four rows)
        const int64_t tiles = g.tilesL * ((g.R + g.Rt - 1) / g.Rt);
        a.rows4 = tiles >= (int64_t)4 * p->num_sms ? 1 : 0;
        a.flags = c.flags;
        a.done = done;
        cudaError_t e = launch_modeprod(1, p->khi(), p->khi(), EPI_RESID, a, g.smem, c.st);
        if (e != cudaSuccess) return e;
        count(c);
    }
    return cudaSuccess;
}

// R = B - sum_j A_j (x)_j X (sigma folded into the first mode) on the tensor
// cores: FP32-pair R in `Rdf` between passes, complex64 R into `Rc64` at the end
// one digit-product pass of mode pass k (tensor cores): out = base -/+ M (x)_j X
cudaError_t run_oz_pass(Ctx &c, size_t k, const unsigned char *img, int eM, const void *X,
                        const void *B, const void *Rin, void *Rout, void *Rc, int in_mode,
                        int out_mode, int neg, float bsign, const int *done) {
    sylv_plan_s *p = c.p;
    const auto &o = p->ozpasses[k];
    OzArgs a{};
    a.X = X;
    a.B = B;
    a.Rin = Rin;
    a.Rout = Rout;
    a.Rc64 = Rc;
    a.in_mode = in_mode;
    a.out_mode = out_mode;
    a.neg = neg;
    a.bsign = bsign;
    a.aimg = img;
    a.n = o.n; a.Kp = o.Kp; a.Np = o.Np; a.mode1 = o.mode1;
    a.lboX = o.lboX; a.sboX = o.sboX; a.sboAd = o.sboAd;
    a.ximg_bytes = o.ximg_bytes; a.aimg_bytes = o.aimg_bytes;
    a.rstage_off = o.rstage_off;
    a.tmem_cols = o.tmem_cols; a.eA = eM;
    a.L = o.L; a.R = o.R; a.tilesL = o.tilesL;
    a.flags = c.flags;
    a.done = done;
    const int64_t tiles = o.mode1 ? (o.R + 63) / 64 : (o.L * o.R + 63) / 64;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, p->num_sms));
    cudaError_t e = launch_resid_oz(a, grid, o.smem, c.st);
    if (e == cudaSuccess) count(c);
    return e;
}

// R = B - sum_j A_j (x)_j X (sigma folded into the first mode) on the tensor
// cores: FP32-pair R in `Rdf` between passes, complex64 R into `Rc64` at the end
cudaError_t run_residual_oz(Ctx &c, const void *B, const void *X, void *Rdf, void *Rc64,
                            const int *done) {
    sylv_plan_s *p = c.p;
    const size_t np = p->ozpasses.size();
    for (size_t k = 0; k < np; ++k) {
        const auto &o = p->ozpasses[k];
        cudaError_t e = run_oz_pass(c, k, o.aimg, o.eA, X, B, Rdf, Rdf, Rc64,
                                    k == 0 ? OZ_IN_B : OZ_IN_PAIRS,
                                    k + 1 == np ? OZ_OUT_C64 : OZ_OUT_PAIRS, 0, 1.f, done);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t run_sweep_cfg(Ctx &c, const SweepConfig &cfg, void *Y, bool fp64) {
    sylv_plan_s *p = c.p;
    SweepArgs a = cfg.a;
    a.Y = Y;
    fill_sweep_ptrs(*p, a, fp64);
    a.cnt = c.cnt;
    a.flags = c.flags;
    cudaError_t e = launch_sweep_init(a, c.st);
    if (e != cudaSuccess) return e;
    count(c);
    e = launch_sweep(fp64, a, cfg.grid, cfg.threads, cfg.smem, c.st);
    if (e != cudaSuccess) return e;
    count(c);
    return cudaSuccess;
}

cudaError_t run_sweep(Ctx &c, void *Y, bool fp64) {
    sylv_plan_s *p = c.p;
    if (!p->diag_sweep) return run_sweep_cfg(c, p->sweep, Y, fp64);
    DiagArgs a = p->diag;
    a.Y = Y;
    a.flags = c.flags;
    cudaError_t e = launch_sweep_diag(fp64, a, p->num_sms, c.st);
    if (e != cudaSuccess) return e;
    count(c);
    return cudaSuccess;
}

sylv_status check_ws(sylv_plan_s *p, void *ws, size_t bytes) {
    if (p->ws_bytes == 0) return SYLV_OK;
    if (!ws || bytes < p->ws_bytes) return SYLV_ERR_WORKSPACE;
    if (((uintptr_t)ws) & 255) return SYLV_ERR_INVALID_ARG;
    return SYLV_OK;
}

sylv_status fill_info(sylv_plan_s *p, DevFlags *flags, cudaStream_t st, sylv_info *info,
                      int launches) {
    DevFlags h{};
    if (cudaMemcpyAsync(&h, flags, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SYLV_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SYLV_ERR_CUDA;
    sylv_status s = SYLV_OK;
    if (h.err & ERRBIT_TIMEOUT) s = SYLV_ERR_TIMEOUT;
    else if (h.err & (ERRBIT_NOTCONV | ERRBIT_NAN)) s = SYLV_ERR_NOT_CONVERGED;
    info->status = s;
    info->refine_iters = p->fp64() ? 0 : h.iters;
    info->launches = launches;
    info->path = (p->diag_sweep ? 1 : 0) | (p->oz ? 2 : 0) | (p->real ? 4 : 0);
    info->last_corr_rel = p->fp64() ? 0.0 : (double)h.lastcorr;
    info->est_rel_err = p->fp64() ? 0.0 : (double)h.est;
    info->min_abs_den = p->min_den;
    info->max_abs_den = p->max_den;
    return s;
}

// A solve is a launch sequence with sweeps between its segments: segment 0
// (init, forward), then for FP64 one sweep and segment 1 (back); for the mixed
// path a sweep before each of segments 1 .. max_refine + 1 (back, refinement
// decision, and -- except in the last -- residual and forward of the next
// correction).  Batched solves interleave equations segment by segment.
int solve_sweeps(const sylv_plan_s *p) { return p->fp64() ? 1 : 1 + p->max_refine; }

// the tensor the sweep after segment `seg` works on
void *sweep_tensor(const sylv_plan_s *p, void *X, void *ws) {
    return p->fp64() ? X : (char *)ws + p->off_W;
}

Ctx make_ctx(sylv_plan_s *p, void *ws, cudaStream_t st) {
    return Ctx{p, st, reinterpret_cast<DevFlags *>(ws),
               reinterpret_cast<int *>((char *)ws + p->off_cnt)};
}

sylv_status solve_segment(Ctx &c, const void *B, void *X, void *ws, int seg) {
    sylv_plan_s *p = c.p;
    cudaStream_t st = c.st;
    cudaError_t e;
    const int KH = p->khi(), KL = p->klo();
    if (p->fp64()) {
        if (seg == 0) {
            if ((e = launch_solve_init(c.flags, st)) != cudaSuccess) return SYLV_ERR_CUDA;
            count(c);
            phase_begin(c, SYLV_PH_FORWARD);
            if (p->Nm == 0) {
                if (B != X && cudaMemcpyAsync(X, B, (size_t)(p->ntot * p->nrhs) * p->ehi(),
                                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                    return SYLV_ERR_CUDA;
            } else if ((e = run_groups(c, p->tgroups, true, 0, B, KH, X, KH, X,
                                       KH, EPI_STORE, nullptr)) != cudaSuccess)
                return SYLV_ERR_CUDA;
            phase_end(c);
        } else {
            phase_begin(c, SYLV_PH_BACK);
            if (p->Nm > 0 && (e = run_groups(c, p->tgroups, true, 1, X, KH, X, KH, X,
                                             KH, EPI_STORE, nullptr)) != cudaSuccess)
                return SYLV_ERR_CUDA;
            phase_end(c);
        }
        return SYLV_OK;
    }
    void *W = (char *)ws + p->off_W;
    void *R = (char *)ws + p->off_R;
    const int *done = &c.flags->done;
    if (seg == 0) {
        // initial low-precision solve X_0: forward of B
        if ((e = launch_solve_init(c.flags, st)) != cudaSuccess) return SYLV_ERR_CUDA;
        count(c);
        phase_begin(c, SYLV_PH_FORWARD);
        if ((e = run_groups(c, p->tgroups, false, 0, B, KH, W, KL, W, KL,
                            EPI_STORE, nullptr)) != cudaSuccess)
            return SYLV_ERR_CUDA;
        phase_end(c);
        return SYLV_OK;
    }
    // back transform of the solve before this segment: X_0 = Y (seg 1) or X += D
    phase_begin(c, SYLV_PH_BACK);
    if (seg == 1 ? run_groups(c, p->tgroups, false, 1, W, KL, W, KL, X, KH,
                              EPI_STORE_NORM, nullptr) != cudaSuccess
                 : run_groups(c, p->tgroups, false, 1, W, KL, W, KL, X, KH,
                              EPI_ACCUM, done) != cudaSuccess)
        return SYLV_ERR_CUDA;
    phase_end(c);
    phase_begin(c, SYLV_PH_UPDATE);
    if (launch_refine_decide(c.flags, (float)p->rtol, seg - 1, p->max_refine, c.st) != cudaSuccess)
        return SYLV_ERR_CUDA;
    count(c);
    phase_end(c);
    if (seg > p->max_refine) return SYLV_OK;
    // correction `seg`: residual and forward transform of it
    phase_begin(c, SYLV_PH_RESIDUAL);
    if (p->oz) {
        // tensor-core residual: complex64 R straight into W
        if (run_residual_oz(c, B, X, R, W, done) != cudaSuccess) return SYLV_ERR_CUDA;
    } else if (run_residual(c, B, X, R, done) != cudaSuccess) {
        return SYLV_ERR_CUDA;
    }
    phase_end(c);
    phase_begin(c, SYLV_PH_FORWARD);
    if (p->oz ? run_groups(c, p->tgroups, false, 0, W, KL, W, KL, W, KL,
                           EPI_STORE, done) != cudaSuccess
              : run_groups(c, p->tgroups, false, 0, R, KH, W, KL, W, KL,
                           EPI_STORE, done) != cudaSuccess)
        return SYLV_ERR_CUDA;
    phase_end(c);
    return SYLV_OK;
}

sylv_status solve_impl(sylv_plan_s *p, const void *B, void *X, void *ws, cudaStream_t st,
                       int &launches) {
    Ctx c = make_ctx(p, ws, st);
    const bool timing = p->timing;
    cudaEvent_t t0 = nullptr;
    if (timing) { t0 = take_event(p); cudaEventRecord(t0, st); }
    const int nsw = solve_sweeps(p);
    for (int seg = 0; seg <= nsw; ++seg) {
        sylv_status s = solve_segment(c, B, X, ws, seg);
        if (s != SYLV_OK) return s;
        if (seg == nsw) break;
        phase_begin(c, SYLV_PH_SWEEP);
        if (run_sweep(c, sweep_tensor(p, X, ws), p->fp64()) != cudaSuccess) return SYLV_ERR_CUDA;
        phase_end(c);
    }
    if (timing) {
        cudaEvent_t t1 = take_event(p);
        cudaEventRecord(t1, st);
        p->tphases.push_back({SYLV_PH_TOTAL, t0, t1, c.launches});
        p->timed_solves++;
    }
    launches = c.launches;
    p->last_launches = c.launches;
    return SYLV_OK;
}

// ------------------------------------------------------ batched graphs --
// One CUDA graph per argument set of sylv_solve_batched: the equations'
// launch sequences spread round-robin over a fork of up to 8 streams.
constexpr int BATCH_STREAMS = 32;
constexpr size_t BATCH_CACHE = 16;

struct BatchGraph {
    std::vector<const void *> key;
    std::vector<int> launches;
    cudaGraphExec_t exec = nullptr;
};

struct DeviceStreams {
    cudaStream_t s[BATCH_STREAMS] = {};
    cudaEvent_t fork = nullptr, join[BATCH_STREAMS] = {};
    bool ready = false;
};

std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch_cache;
DeviceStreams g_dev_streams[64];

// drop the recorded graphs that reference plan p (its tables changed or died)
void batch_forget(const void *p) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batch_cache.size();) {
        const auto &k = g_batch_cache[i].key;
        bool hit = false;
        for (size_t q = 2; q < k.size(); q += 3) hit |= (k[q] == p);
        if (hit) {
            cudaGraphExecDestroy(g_batch_cache[i].exec);
            g_batch_cache.erase(g_batch_cache.begin() + (long)i);
        } else {
            ++i;
        }
    }
}

// One segment's sweeps of the equations `eqs` (tiled sweeps): grouped by
// kernel template and block size, each group in chunks of at most SWB_MAX
// equations, one persistent launch per chunk (k_sweep_batch) on `st`.  Larger
// equations first, so that the CTAs' work-weighted starts spread over them.
cudaError_t run_sweep_batched(const sylv_plan_t *plans, void *const *X, void *ws,
                              const std::vector<size_t> &off, const std::vector<int> &eqs,
                              cudaStream_t st, std::vector<Ctx> &ctx) {
    std::vector<int> order(eqs);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const sylv_plan_s *a = plans[x], *b = plans[y];
        const int ka = (a->fp64() ? 4 : 0) + (a->real ? 2 : 0), kb = (b->fp64() ? 4 : 0) + (b->real ? 2 : 0);
        if (ka != kb) return ka < kb;
        if (a->sweep.threads != b->sweep.threads) return a->sweep.threads < b->sweep.threads;
        return a->sweep.a.ntiles > b->sweep.a.ntiles;
    });
    auto same = [&](int x, int y) {
        const sylv_plan_s *a = plans[x], *b = plans[y];
        return a->fp64() == b->fp64() && a->real == b->real && a->sweep.threads == b->sweep.threads;
    };
    std::unique_ptr<SweepBatch> bt(new (std::nothrow) SweepBatch);
    if (!bt) return cudaErrorMemoryAllocation;
    const int num_sms = plans[order[0]]->num_sms;
    for (size_t i = 0; i < order.size();) {
        size_t j = i;
        while (j < order.size() && j - i < (size_t)SWB_MAX && same(order[i], order[j])) ++j;
        std::memset(bt.get(), 0, sizeof(SweepBatch));
        bt->neq = (int)(j - i);
        bt->far_split = bt->neq == 1 ? 1 : 0;
        size_t smem = 0;
        long long cum = 0;
        for (size_t q = i; q < j; ++q) {
            const int e = order[q];
            sylv_plan_s *p = plans[e];
            const int k = (int)(q - i);
            bt->sa[k] = p->sweep.dargs;
            bt->Y[k] = sweep_tensor(p, X[e], (char *)ws + off[(size_t)e]);
            bt->cnt[k] = reinterpret_cast<int *>((char *)ws + off[(size_t)e] + p->off_cnt);
            bt->flags[k] = reinterpret_cast<DevFlags *>((char *)ws + off[(size_t)e]);
            bt->cum[k] = cum;
            cum += p->sweep.a.ntiles;
            smem = std::max(smem, p->sweep.smem);
            ctx[(size_t)e].launches += 2;
        }
        bt->cum[bt->neq] = cum;
        const sylv_plan_s *p0 = plans[order[i]];
        const int threads = p0->sweep.threads;
        int per = sweep_batch_blocks_per_sm(p0->fp64(), threads, smem, p0->real ? 1 : 0);
        if (per < 1) per = 1;
        const int grid = (int)std::max<long long>(1, std::min<long long>((long long)num_sms * per, cum));
        cudaError_t e = launch_sweep_batch(p0->fp64(), p0->real ? 1 : 0, *bt, grid, threads, smem, st);
        if (e != cudaSuccess) return e;
        i = j;
    }
    return cudaSuccess;
}

sylv_status batch_graph_launch(int count, const sylv_plan_t *plans, const void *const *B,
                               void *const *X, void *ws, cudaStream_t user,
                               std::vector<int> &launches) {
    const int dev = plans[0]->device;
    if (dev < 0 || dev >= 64) return SYLV_ERR_INVALID_ARG;
    std::vector<const void *> key;
    key.reserve(3 * (size_t)count + 2);
    key.push_back(ws);
    key.push_back(reinterpret_cast<const void *>((uintptr_t)count));
    for (int e = 0; e < count; ++e) {
        key.push_back(plans[e]);
        key.push_back(B[e]);
        key.push_back(X[e]);
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto &g : g_batch_cache)
        if (g.key == key) {
            launches = g.launches;
            return cudaGraphLaunch(g.exec, user) == cudaSuccess ? SYLV_OK : SYLV_ERR_CUDA;
        }
    DeviceStreams &ds = g_dev_streams[dev];
    if (!ds.ready) {
        for (int k = 0; k < BATCH_STREAMS; ++k)
            if (cudaStreamCreateWithFlags(&ds.s[k], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ds.join[k], cudaEventDisableTiming) != cudaSuccess)
                return SYLV_ERR_CUDA;
        if (cudaEventCreateWithFlags(&ds.fork, cudaEventDisableTiming) != cudaSuccess)
            return SYLV_ERR_CUDA;
        ds.ready = true;
    }
    const int S = std::min(count, BATCH_STREAMS);
    cudaStream_t cs = ds.s[0];
    std::vector<size_t> off((size_t)count, 0);
    for (int e = 1; e < count; ++e) off[(size_t)e] = off[(size_t)e - 1] + align256(plans[e - 1]->ws_bytes);
    std::vector<Ctx> ctx;
    ctx.reserve((size_t)count);
    int maxsw = 0;
    for (int e = 0; e < count; ++e) {
        ctx.push_back(make_ctx(plans[e], (char *)ws + off[(size_t)e], ds.s[e % S]));
        maxsw = std::max(maxsw, solve_sweeps(plans[e]));
    }
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return SYLV_ERR_CUDA;
    bool ok = cudaEventRecord(ds.fork, cs) == cudaSuccess;
    for (int k = 1; ok && k < S; ++k) ok = cudaStreamWaitEvent(ds.s[k], ds.fork, 0) == cudaSuccess;
    // segment by segment: every equation's launches up to its next sweep on its
    // stream; then one batched sweep over the equations with tiled sweeps (the
    // entrywise-division sweeps of Remark 1 stay on their own streams)
    for (int seg = 0; ok && seg <= maxsw; ++seg) {
        std::vector<int> tiled;
        for (int e = 0; ok && e < count; ++e) {
            sylv_plan_s *p = plans[e];
            const int nsw = solve_sweeps(p);
            if (seg > nsw) continue;
            ok = solve_segment(ctx[(size_t)e], B[e], X[e], (char *)ws + off[(size_t)e], seg) ==
                 SYLV_OK;
            if (!ok || seg == nsw) continue;
            if (p->diag_sweep || p->Nm == 0)
                ok = run_sweep(ctx[(size_t)e], sweep_tensor(p, X[e], (char *)ws + off[(size_t)e]),
                               p->fp64()) == cudaSuccess;
            else
                tiled.push_back(e);
        }
        if (!ok || tiled.empty()) continue;
        for (int k = 1; ok && k < S; ++k)
            ok = cudaEventRecord(ds.join[k], ds.s[k]) == cudaSuccess &&
                 cudaStreamWaitEvent(cs, ds.join[k], 0) == cudaSuccess;
        if (ok) ok = run_sweep_batched(plans, X, ws, off, tiled, cs, ctx) == cudaSuccess;
        if (ok) ok = cudaEventRecord(ds.fork, cs) == cudaSuccess;
        for (int k = 1; ok && k < S; ++k) ok = cudaStreamWaitEvent(ds.s[k], ds.fork, 0) == cudaSuccess;
    }
    for (int e = 0; e < count; ++e) launches[(size_t)e] = ctx[(size_t)e].launches;
    for (int k = 1; ok && k < S; ++k)
        ok = cudaEventRecord(ds.join[k], ds.s[k]) == cudaSuccess &&
             cudaStreamWaitEvent(cs, ds.join[k], 0) == cudaSuccess;
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (!ok || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return SYLV_ERR_CUDA;
    }
    BatchGraph bg;
    bg.key = std::move(key);
    bg.launches = launches;
    ec = cudaGraphInstantiate(&bg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) return SYLV_ERR_CUDA;
    if (g_batch_cache.size() >= BATCH_CACHE) {
        cudaGraphExecDestroy(g_batch_cache.front().exec);
        g_batch_cache.erase(g_batch_cache.begin());
    }
    g_batch_cache.push_back(std::move(bg));
    return cudaGraphLaunch(g_batch_cache.back().exec, user) == cudaSuccess ? SYLV_OK
                                                                           : SYLV_ERR_CUDA;
}

}  // namespace

// ===================================================================== ABI ==

extern "C" {

int sylv_version(void) { return 100; }

const char *sylv_status_string(sylv_status s) {
    switch (s) {
        case SYLV_OK: return "ok";
        case SYLV_ERR_INVALID_ARG: return "invalid argument";
        case SYLV_ERR_SHAPE: return "unsupported shape";
        case SYLV_ERR_SINGULAR: return "singular: a diagonal sum t_1+...+t_N is zero or not finite";
        case SYLV_ERR_NOT_CONVERGED: return "refinement did not converge";
        case SYLV_ERR_TIMEOUT: return "device dependency wait timed out";
        case SYLV_ERR_OOM: return "device allocation failed";
        case SYLV_ERR_CUDA: return "CUDA error";
        case SYLV_ERR_SCHUR: return "Schur iteration did not converge";
        case SYLV_ERR_WORKSPACE: return "workspace missing or too small";
    }
    return "unknown status";
}

sylv_status sylv_schur(int64_t n, const double *A, double *Q, double *T) {
    if (n < 1 || n > MAX_N) return SYLV_ERR_SHAPE;
    try {
        return schur_host(n, A, Q, T);
    } catch (...) {
        return SYLV_ERR_OOM;
    }
}

sylv_status sylv_expm(int64_t n, const double *M, double *E) {
    if (!M || !E) return SYLV_ERR_INVALID_ARG;
    if (n < 1 || n > MAX_N) return SYLV_ERR_SHAPE;
    try {
        return expm_host(n, M, E);
    } catch (...) {
        return SYLV_ERR_OOM;
    }
}

// The 2 x 2 blocks of a real quasi-triangular T (at even offsets) rotated to
// complex triangular form: V = [u1 u2] with u1 the unit eigenvector of the
// block's eigenvalue lambda (positive imaginary part) and u2 = (-conj(u1[1]),
// conj(u1[0])), so V^* B V = [lambda *; 0 conj(lambda)].  Returns V (4 complex
// entries per index pair, identity for pairs of 1 x 1 blocks) and
// Tt = V^* T V with its rounding-level entries below the diagonal cleared.
static bool rotate_quasi_triangular(int64_t n, const std::vector<double> &T, std::vector<cd> &V,
                             std::vector<cd> &Tt, bool &pairs) {
    const int64_t np = (n + 1) / 2;
    V.assign((size_t)(4 * np), cd(0.0));
    pairs = false;
    for (int64_t u = 0; u < np; ++u) {
        cd *v = V.data() + 4 * u;
        const int64_t k = 2 * u;
        if (k + 1 < n && T[(size_t)(k + 1 + k * n)] != 0.0) {
            const double a = T[(size_t)(k + k * n)], b = T[(size_t)(k + (k + 1) * n)];
            const double c = T[(size_t)(k + 1 + k * n)], d = T[(size_t)(k + 1 + (k + 1) * n)];
            const double p = 0.5 * (a - d), disc = p * p + b * c;
            if (!(disc < 0.0) || b == 0.0) return false;
            const cd lam(0.5 * (a + d), std::sqrt(-disc));
            cd x = b, y = lam - a;
            const double h = std::sqrt(std::norm(x) + std::norm(y));
            x /= h;
            y /= h;
            v[0] = x; v[1] = y; v[2] = -std::conj(y); v[3] = std::conj(x);
            pairs = true;
        } else {
            v[0] = 1.0; v[3] = 1.0;
        }
    }
    // Tt = V^* T V, V block diagonal: Tt[r, c] = sum over the blocks of r and c
    Tt.assign((size_t)(n * n), cd(0.0));
    auto Vat = [&](int64_t r, int64_t c) -> cd {   // V[r, c], zero off the 2 x 2 blocks
        if (r / 2 != c / 2) return cd(0.0);
        const cd *v = V.data() + 4 * (r / 2);
        return v[(r & 1) + 2 * (c & 1)];
    };
    for (int64_t c = 0; c < n; ++c)
        for (int64_t r = 0; r < n; ++r) {
            cd sum = 0.0;
            for (int64_t rr = r & ~1LL; rr < std::min<int64_t>(n, (r & ~1LL) + 2); ++rr)
                for (int64_t cc = c & ~1LL; cc < std::min<int64_t>(n, (c & ~1LL) + 2); ++cc)
                    sum += std::conj(Vat(rr, r)) * T[(size_t)(rr + cc * n)] * Vat(cc, c);
            Tt[(size_t)(r + c * n)] = sum;
        }
    double nrm = 0.0;
    for (double t : T) nrm = std::max(nrm, std::fabs(t));
    for (int64_t c = 0; c < n; ++c)
        for (int64_t r = c + 1; r < n; ++r) {
            if (std::abs(Tt[(size_t)(r + c * n)]) > 1e-12 * std::max(nrm, 1e-300)) return false;
            Tt[(size_t)(r + c * n)] = 0.0;
        }
    return true;
}

static sylv_status create_plan(sylv_plan_t *out, int N, const int64_t *n, int64_t nrhs,
                               const double *const *A, const double *const *Q,
                               const double *const *T, const double *const *Areal, int prec,
                               double rtol, int max_refine, int device,
                               const sylv_tuning *tuning) {
    if (!out) return SYLV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!n || N < 1 || N > 256 || nrhs < 1) return SYLV_ERR_SHAPE;
    if (prec != SYLV_FP64 && prec != SYLV_MIXED_FP32 && prec != SYLV_MIXED_FP32_EMU)
        return SYLV_ERR_INVALID_ARG;
    const bool real = Areal != nullptr;
    if (real && prec == SYLV_MIXED_FP32_EMU) return SYLV_ERR_INVALID_ARG;
    const bool haveA = A != nullptr, haveQT = (Q != nullptr && T != nullptr);
    if (real ? (haveA || haveQT) : (haveA == haveQT)) return SYLV_ERR_INVALID_ARG;
    if (prec != SYLV_FP64 && (!(rtol > 0.0) || max_refine < 1)) return SYLV_ERR_INVALID_ARG;
    sylv_plan_s *p = nullptr;
    try {
        p = new sylv_plan_s();
    } catch (...) {
        return SYLV_ERR_OOM;
    }
    std::unique_ptr<sylv_plan_s> guard(p);
    p->device = device;
    p->prec = prec;
    p->rtol = rtol;
    p->max_refine = max_refine;
    p->N_in = N;
    p->nrhs = nrhs;
    p->n_in.assign(n, n + N);
    p->real = real;
    // shapes, strides, overflow
    int64_t tot = 1;
    for (int j = 0; j < N; ++j) {
        if (n[j] < 1 || n[j] > MAX_N) return SYLV_ERR_SHAPE;
        if (tot > (int64_t)(INT64_MAX / 16) / n[j]) return SYLV_ERR_SHAPE;
        if (n[j] > 1) {
            if (p->Nm >= MAXM) return SYLV_ERR_SHAPE;
            p->n[p->Nm] = n[j];
            p->S[p->Nm] = tot;
            p->orig[p->Nm] = j;
            p->Nm++;
        }
        tot *= n[j];
    }
    if (tot > (int64_t)(INT64_MAX / 16) / nrhs) return SYLV_ERR_SHAPE;
    p->ntot = tot;

    // factors on the host
    p->Ah.resize(N);
    p->Qh.resize(N);
    p->Th.resize(N);
    if (real) {
        p->Qr.resize(N);
        p->Tr.resize(N);
        p->Vh.resize(N);
    }
    for (int j = 0, jm = 0; j < N; ++j) {
        const int64_t nj = n[j], nn = nj * nj;
        auto &Aj = p->Ah[j];
        auto &Qj = p->Qh[j];
        auto &Tj = p->Th[j];
        Aj.assign((size_t)nn, 0.0);
        Qj.assign((size_t)nn, 0.0);
        Tj.assign((size_t)nn, 0.0);
        if (real) {
            // A_j = Q_j T_j Q_j^T (real Schur, 2 x 2 blocks at even offsets), and
            // the complex triangular T~_j = V_j^* T_j V_j the sweep uses in a tile
            if (!Areal[j]) return SYLV_ERR_INVALID_ARG;
            auto &Qr = p->Qr[j];
            auto &Tr = p->Tr[j];
            Qr.assign((size_t)nn, 0.0);
            Tr.assign((size_t)nn, 0.0);
            for (int64_t k = 0; k < nn; ++k) Aj[(size_t)k] = cd(Areal[j][k], 0.0);
            if (nj == 1) {
                Qr[0] = 1.0;
                Tr[0] = Areal[j][0];
                Qj[0] = 1.0;
                Tj[0] = Aj[0];
            } else {
                sylv_status s = schur_real_host(nj, Areal[j], Qr.data(), Tr.data());
                if (s != SYLV_OK) return s;
                bool pairs = false;
                if (!rotate_quasi_triangular(nj, Tr, p->Vh[j], Tj, pairs)) return SYLV_ERR_SCHUR;
                for (int64_t k = 0; k < nn; ++k) Qj[(size_t)k] = Qr[(size_t)k];
                p->has_pairs[jm] = pairs;
            }
        } else if (haveA) {
            if (!A[j]) return SYLV_ERR_INVALID_ARG;
            for (int64_t k = 0; k < nn; ++k) Aj[(size_t)k] = cd(A[j][2 * k], A[j][2 * k + 1]);
            if (nj == 1) {
                Qj[0] = 1.0;
                Tj[0] = Aj[0];
            } else {
                std::vector<double> q((size_t)(2 * nn)), t((size_t)(2 * nn));
                sylv_status s = schur_host(nj, A[j], q.data(), t.data());
                if (s != SYLV_OK) return s;
                for (int64_t k = 0; k < nn; ++k) {
                    Qj[(size_t)k] = cd(q[2 * k], q[2 * k + 1]);
                    Tj[(size_t)k] = cd(t[2 * k], t[2 * k + 1]);
                }
            }
        } else {
            if (!T[j] || (nj > 1 && !Q[j])) return SYLV_ERR_INVALID_ARG;
            for (int64_t c = 0; c < nj; ++c)
                for (int64_t r = 0; r < nj; ++r) {
                    int64_t k = r + c * nj;
                    Tj[(size_t)k] = r <= c ? cd(T[j][2 * k], T[j][2 * k + 1]) : cd(0.0, 0.0);
                    Qj[(size_t)k] = nj == 1 ? cd(1.0, 0.0) : cd(Q[j][2 * k], Q[j][2 * k + 1]);
                }
            // A = Q T Q^*
            for (int64_t c = 0; c < nj; ++c)
                for (int64_t r = 0; r < nj; ++r) {
                    cd s = 0.0;
                    for (int64_t a = 0; a < nj; ++a)
                        for (int64_t b = a; b < nj; ++b)
                            s += Qj[(size_t)(r + a * nj)] * Tj[(size_t)(a + b * nj)] *
                                 std::conj(Qj[(size_t)(c + b * nj)]);
                    Aj[(size_t)(r + c * nj)] = s;
                }
        }
        for (auto &z : Tj)
            if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) return SYLV_ERR_INVALID_ARG;
        if (nj == 1) p->sigma += Tj[0];
        if (nj > 1) ++jm;
    }
    // Remark 1: when every A_j is normal its Schur factor T_j is diagonal up
    // to rounding (||strict upper||_F of order n_j u ||T_j||_F); dropping that
    // part perturbs A_j at the level of the Schur step's own backward error,
    // and the sweep becomes an entrywise division
    if (!(tuning && tuning->general_sweep) && p->Nm > 0 && !real) {
        bool diag = true;
        for (int j = 0; diag && j < p->Nm; ++j) {
            const auto &Tj = p->Th[p->orig[j]];
            const int64_t nj = p->n[j];
            double off = 0.0, all = 0.0;
            for (int64_t c = 0; c < nj; ++c)
                for (int64_t r = 0; r <= c; ++r) {
                    const double a2 = std::norm(Tj[(size_t)(r + c * nj)]);
                    all += a2;
                    if (r < c) off += a2;
                }
            diag = std::sqrt(off) <= 4.0 * (double)nj * std::ldexp(1.0, -53) * std::sqrt(all);
        }
        p->diag_sweep = diag;
    }
    int diag_h = 0;
    int64_t diag_P1 = 1;
    if (p->diag_sweep) {
        diag_P1 = p->n[0];
        diag_h = 1;
        while (diag_h < p->Nm && diag_P1 * p->n[diag_h] <= DIAG_HEAD_MAX) diag_P1 *= p->n[diag_h++];
    }

    // device
    {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
            return SYLV_ERR_CUDA;
    }
    DeviceGuard dg(device);
    if (!dg.ok) return SYLV_ERR_CUDA;
    if (ensure_init(device) != SYLV_OK) return SYLV_ERR_CUDA;
    {
        int sms = 0, khz = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
        p->num_sms = std::max(1, sms);
        const long long ms = (tuning && tuning->timeout_ms > 0) ? tuning->timeout_ms : 2000;
        p->timeout_cycles = ms * (long long)std::max(khz, 1000000);
        p->fault_tile = (tuning && tuning->fault_tile > 0) ? tuning->fault_tile - 1 : -1;
    }

    // transform and residual passes
    const int gmax = tuning ? tuning->group_max : 0;
    const bool allow_tc = !(tuning && tuning->no_tensor_cores);
    p->tc_plain = tuning && tuning->tc_plain;
    p->tgroup_max = gmax;
    sylv_status s = make_groups(*p, p->fp64(), true, gmax, allow_tc, p->tgroups);
    if (s != SYLV_OK) return s;
    s = make_groups(*p, true, false, gmax, false, p->rgroups);
    if (s != SYLV_OK) return s;
    if (p->emu()) p->oz = make_oz_passes(*p, p->ozpasses);
    if (p->fp64() || real) {          // (no Theorem 1 passes for a real plan)
        p->egroups = p->tgroups;
    } else {
        s = make_groups(*p, true, true, gmax, false, p->egroups);
        if (s != SYLV_OK) return s;
    }
    // device pool: per mode Uh64 U64 A64 T64 d64 Uh32 U32 T32, then the tables
    size_t off = 0;
    std::vector<size_t> offs;
    auto reserve = [&](size_t bytes) { off = align256(off); offs.push_back(off); off += bytes; };
    for (int j = 0; j < p->Nm; ++j) {
        size_t nn = (size_t)(p->n[j] * p->n[j]);
        // the FP64 product matrices (U_j^*, U_j, A_j, -A_j, exp(t A_j)) carry a
        // plane re + im after the complex entries (three-multiplication products)
        reserve(nn * 24); reserve(nn * 24); reserve(nn * 24); reserve(nn * 16);
        reserve((size_t)p->n[j] * 16);
        reserve(nn * 8); reserve(nn * 8); reserve(nn * 8);
        reserve(nn * 24); reserve(nn * 24);              // -A_j, exp(t A_j)
        // real variant: T_j (FP64, FP32) and the pair rotations V_j (FP64, FP32)
        const size_t np = (size_t)((p->n[j] + 1) / 2) * 4;
        reserve(p->real ? nn * 8 : 0); reserve(p->real ? nn * 4 : 0);
        reserve(p->real ? np * 16 : 0); reserve(p->real ? np * 8 : 0);
    }
    reserve(3 * sizeof(unsigned long long));
    const size_t oz_first = offs.size();
    if (p->oz)
        for (auto &o : p->ozpasses) {
            reserve((size_t)6 * o.aimg_bytes);     // A digits
            reserve((size_t)6 * o.aimg_bytes);     // exp(t A) digits, filled by sylv_evolve
        }
    const size_t diag_idx = offs.size();
    if (p->diag_sweep) reserve((size_t)diag_P1 * 16);
    const size_t tc_first = offs.size();
    for (auto &g : p->tgroups)
        if (g.tc) {
            reserve((size_t)2 * g.bimg_bytes);     // U^*: hi, lo
            reserve((size_t)2 * g.bimg_bytes);     // U: hi, lo
        }
    size_t pool_bytes = align256(off);
    if (cudaMalloc(&p->dpool, pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        return SYLV_ERR_OOM;
    }
    std::vector<char> host(pool_bytes, 0);
    size_t oi = 0;
    char *base = (char *)p->dpool;
    for (int j = 0; j < p->Nm; ++j) {
        const int jj = p->orig[j];
        const int64_t nj = p->n[j];
        const auto &Qj = p->Qh[jj];
        const auto &Tj = p->Th[jj];
        const auto &Aj = p->Ah[jj];
        double *uh64 = (double *)(host.data() + offs[oi]);
        double *u64 = (double *)(host.data() + offs[oi + 1]);
        double *a64 = (double *)(host.data() + offs[oi + 2]);
        double *t64 = (double *)(host.data() + offs[oi + 3]);
        double *d64 = (double *)(host.data() + offs[oi + 4]);
        float *uh32 = (float *)(host.data() + offs[oi + 5]);
        float *u32 = (float *)(host.data() + offs[oi + 6]);
        float *t32 = (float *)(host.data() + offs[oi + 7]);
        for (int64_t c = 0; p->real && c < nj; ++c)
            for (int64_t r = 0; r < nj; ++r) {
                // real tensors: Q^T, Q, A as plain float64 / float32 matrices; the
                // sweep's T~_j complex as for the complex plan
                const size_t k = (size_t)(r + c * nj);
                const double qt = p->Qr[jj][(size_t)(c + r * nj)], q = p->Qr[jj][k];
                uh64[k] = qt;
                u64[k] = q;
                a64[k] = Aj[k].real();
                uh32[k] = (float)qt;
                u32[k] = (float)q;
                t64[2 * k] = Tj[k].real(); t64[2 * k + 1] = Tj[k].imag();
                t32[2 * k] = (float)Tj[k].real(); t32[2 * k + 1] = (float)Tj[k].imag();
                ((double *)(host.data() + offs[oi + 10]))[k] = p->Tr[jj][k];
                ((float *)(host.data() + offs[oi + 11]))[k] = (float)p->Tr[jj][k];
            }
        if (p->real) {
            const auto &V = p->Vh[jj];
            double *v64 = (double *)(host.data() + offs[oi + 12]);
            float *v32 = (float *)(host.data() + offs[oi + 13]);
            for (size_t k = 0; k < V.size(); ++k) {
                v64[2 * k] = V[k].real(); v64[2 * k + 1] = V[k].imag();
                v32[2 * k] = (float)V[k].real(); v32[2 * k + 1] = (float)V[k].imag();
            }
            p->Tr64[j] = base + offs[oi + 10];
            p->Tr32[j] = base + offs[oi + 11];
            p->V64[j] = base + offs[oi + 12];
            p->V32[j] = base + offs[oi + 13];
        }
        for (int64_t c = 0; !p->real && c < nj; ++c)
            for (int64_t r = 0; r < nj; ++r) {
                size_t k = (size_t)(r + c * nj);
                cd uh = std::conj(Qj[(size_t)(c + r * nj)]);   // (U^*)[r, c]
                cd u = Qj[k];
                uh64[2 * k] = uh.real(); uh64[2 * k + 1] = uh.imag();
                u64[2 * k] = u.real(); u64[2 * k + 1] = u.imag();
                a64[2 * k] = Aj[k].real(); a64[2 * k + 1] = Aj[k].imag();
                t64[2 * k] = Tj[k].real(); t64[2 * k + 1] = Tj[k].imag();
                uh32[2 * k] = (float)uh.real(); uh32[2 * k + 1] = (float)uh.imag();
                u32[2 * k] = (float)u.real(); u32[2 * k + 1] = (float)u.imag();
                t32[2 * k] = (float)Tj[k].real(); t32[2 * k + 1] = (float)Tj[k].imag();
            }
        for (int64_t i = 0; i < nj; ++i) {
            d64[2 * i] = Tj[(size_t)(i + i * nj)].real();
            d64[2 * i + 1] = Tj[(size_t)(i + i * nj)].imag();
        }
        p->Uh64[j] = base + offs[oi];
        p->U64[j] = base + offs[oi + 1];
        p->A64[j] = base + offs[oi + 2];
        p->T64[j] = base + offs[oi + 3];
        p->d64[j] = (const double *)(base + offs[oi + 4]);
        p->Uh32[j] = base + offs[oi + 5];
        p->U32[j] = base + offs[oi + 6];
        p->T32[j] = base + offs[oi + 7];
        double *na64 = (double *)(host.data() + offs[oi + 8]);
        for (size_t k = 0; !p->real && k < (size_t)(2 * nj * nj); ++k) na64[k] = -a64[k];
        for (size_t k = 0; !p->real && k < (size_t)(nj * nj); ++k) {
            uh64[2 * nj * nj + k] = uh64[2 * k] + uh64[2 * k + 1];
            u64[2 * nj * nj + k] = u64[2 * k] + u64[2 * k + 1];
            a64[2 * nj * nj + k] = a64[2 * k] + a64[2 * k + 1];
            na64[2 * nj * nj + k] = na64[2 * k] + na64[2 * k + 1];
        }
        p->nA64[j] = base + offs[oi + 8];
        p->E64[j] = base + offs[oi + 9];
        oi += 14;
    }
    unsigned long long *dm = (unsigned long long *)(base + offs[oi]);
    unsigned long long init3[3] = {~0ull, 0ull, 0ull};
    std::memcpy(host.data() + offs[oi], init3, sizeof(init3));
    // tensor-core B operands: B[k, i] = Re M[i, k], B[k, n + i] = Im M[i, k]
    // (M = U^* forward, U back), split into TF32 hi and lo, in the K-major
    // no-swizzle layout the kernel's descriptors describe
    {
        size_t ti = tc_first;
        for (auto &g : p->tgroups) {
            if (!g.tc) continue;
            const int j = g.first, n = (int)p->n[j];
            const auto &Qj = p->Qh[p->orig[j]];
            for (int dir = 0; dir < 2; ++dir) {
                unsigned char *hi = reinterpret_cast<unsigned char *>(host.data()) + offs[ti + dir];
                unsigned char *lo = hi + g.bimg_bytes;
                for (int ii = 0; ii < g.Np; ++ii)
                    for (int k = 0; k < g.Kp; ++k) {
                        float v = 0.f;
                        if (k < n && ii < 2 * n) {
                            const int i = ii < n ? ii : ii - n;
                            const cd m = dir == 0 ? std::conj(Qj[(size_t)(k + i * n)])
                                                  : Qj[(size_t)(i + k * n)];
                            v = (float)(ii < n ? m.real() : m.imag());
                        }
                        uint32_t u;
                        std::memcpy(&u, &v, 4);
                        if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
                        float h;
                        std::memcpy(&h, &u, 4);
                        const float l = v - h;
                        const size_t off = (size_t)(ii / 8) * g.sboB + (size_t)(k / 4) * 128 +
                                           (size_t)(ii % 8) * 16 + (size_t)(k % 4) * 4;
                        std::memcpy(hi + off, &h, 4);
                        std::memcpy(lo + off, &l, 4);
                    }
                g.img[dir] = (const unsigned char *)(base + offs[ti + dir]);
            }
            ti += 2;
        }
    }
    // residual digit images: [Re A^T | Im A^T] of A_j (A_1 + sigma I for the
    // first mode) as 6 base-256 digits of |a| / 2^eA, bf16, K-major layout
    if (p->oz) {
        size_t oi2 = oz_first;
        for (auto &o : p->ozpasses) {
            const int j = o.j, n = o.n;
            std::vector<cd> Am(p->Ah[p->orig[j]]);
            if (j == 0)
                for (int i = 0; i < n; ++i) Am[(size_t)(i + i * n)] += p->sigma;
            unsigned char *img = reinterpret_cast<unsigned char *>(host.data()) + offs[oi2];
            o.eA = digit_images(Am, o, img);
            o.aimg = (const unsigned char *)(base + offs[oi2]);
            o.eimg = (const unsigned char *)(base + offs[oi2 + 1]);
            oi2 += 2;
        }
    }
    // diagonal-sweep head table: sigma + sum of t_{j,i_j i_j} over the head modes
    if (p->diag_sweep) {
        double *tab = (double *)(host.data() + offs[diag_idx]);
        for (int64_t q = 0; q < diag_P1; ++q) {
            cd sum = p->sigma;
            int64_t r = q;
            for (int j = 0; j < diag_h; ++j) {
                const int64_t i = r % p->n[j];
                r /= p->n[j];
                sum += p->Th[p->orig[j]][(size_t)(i + i * p->n[j])];
            }
            tab[2 * q] = sum.real();
            tab[2 * q + 1] = sum.imag();
        }
        DiagArgs &d = p->diag;
        d.total = p->ntot * p->nrhs;
        d.P1 = diag_P1;
        d.Qt = p->ntot / diag_P1;
        d.dhead = (const double *)(base + offs[diag_idx]);
        d.Nt = p->Nm - diag_h;
        for (int m = 0; m < d.Nt; ++m) {
            d.tn[m] = p->n[diag_h + m];
            d.td[m] = p->d64[diag_h + m];
        }
    }
    if (cudaMemcpy(p->dpool, host.data(), pool_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return SYLV_ERR_CUDA;

    // diagonal sums: min / max |sigma + sum_j t_{j,i_j i_j}|
    if (launch_den_minmax(p->Nm, p->n, p->d64, p->sigma.real(), p->sigma.imag(), p->ntot, dm,
                          0) != cudaSuccess)
        return SYLV_ERR_CUDA;
    unsigned long long r3[3];
    if (cudaMemcpy(r3, dm, sizeof(r3), cudaMemcpyDeviceToHost) != cudaSuccess) return SYLV_ERR_CUDA;
    double mn, mx;
    std::memcpy(&mn, &r3[0], 8);
    std::memcpy(&mx, &r3[1], 8);
    p->min_den = mn;
    p->max_den = mx;
    if (r3[2] != 0 || !(mn > 0.0) || !std::isfinite(mx)) return SYLV_ERR_SINGULAR;
    // power of two centring |scale * sum|^2 on 1 for the sweep's reciprocals
    p->den_scale = std::ldexp(1.0, -(int)std::lround(0.5 * (std::log2(mn) + std::log2(mx))));
    p->diag.den_scale = p->den_scale;
    // the tensor-core residual is accurate to ~2^-45 of sum_j ||A_j|| ||X||, so the
    // refined solution's error is about kappa 2^-45; keep it only when the
    // eigenvalue-sum ratio (a lower bound of kappa) leaves a margin below rtol
    if (p->oz && (mx / mn) * std::ldexp(1.0, -44) > p->rtol) p->oz = false;
    // the sweep's reciprocals, once per plan, when the table stays within budget
    if (!p->diag_sweep && p->Nm > 0 && (size_t)p->ntot * 16 <= INV_TABLE_MAX) {
        if (cudaMalloc(&p->inv_tab, (size_t)p->ntot * 16) != cudaSuccess) {
            cudaGetLastError();
            p->inv_tab = nullptr;            // fall back to forming them in the sweep
        } else {
            SweepArgs ta{};
            ta.Nm = p->Nm;
            for (int j = 0; j < p->Nm; ++j) { ta.n[j] = p->n[j]; ta.d[j] = p->d64[j]; }
            ta.sig_re = p->sigma.real();
            ta.sig_im = p->sigma.imag();
            ta.ntot = p->ntot;
            ta.den_scale = p->den_scale;
            if (launch_inv_table(p->fp64(), ta, p->inv_tab, p->num_sms, 0) != cudaSuccess ||
                cudaDeviceSynchronize() != cudaSuccess)
                return SYLV_ERR_CUDA;
        }
    }

    // sweep: default tiles (FP64 256 entries x 128 threads, FP32 1024 x 256,
    // measured on GB300) or the caller's block extents
    {
        int b[MAXM];
        choose_blocks(*p, p->fp64() ? 256 : 1024, tuning, b);
        int threads = p->fp64() ? 128 : 256;
        if (tuning && tuning->sweep_threads > 0)
            threads = std::min(256, (tuning->sweep_threads + 31) / 32 * 32);
        s = build_sweep(*p, b, threads, p->sweep, tuning ? tuning->sweep_ctas_per_sm : 0);
        if (s != SYLV_OK) return s;
        // tile counters for any tiling the autotuner may install (tiles >= 64 entries)
        p->cnt_capacity = p->sweep.a.ntiles;
        for (int target = 64; target <= 4096; target *= 2) {
            int bt[MAXM];
            choose_blocks(*p, target, nullptr, bt);
            p->cnt_capacity = std::max(p->cnt_capacity, tiles_for(*p, bt));
        }
    }

    // workspace layout
    size_t w = align256(sizeof(DevFlags));
    p->off_cnt = w;
    w = align256(w + (size_t)p->cnt_capacity * 4);
    if (!p->fp64()) {
        p->off_W = w;
        w = align256(w + (size_t)(p->ntot * p->nrhs) * p->elo());
        p->off_R = w;
        w = align256(w + (size_t)(p->ntot * p->nrhs) * p->ehi());
    }
    p->ws_bytes = w;
    *out = guard.release();
    return SYLV_OK;
}

sylv_status sylv_plan_create(sylv_plan_t *out, int N, const int64_t *n, int64_t nrhs,
                             const double *const *A, const double *const *Q,
                             const double *const *T, int prec, double rtol, int max_refine,
                             int device, const sylv_tuning *tuning) {
    return create_plan(out, N, n, nrhs, A, Q, T, nullptr, prec, rtol, max_refine, device, tuning);
}

sylv_status sylv_plan_create_real(sylv_plan_t *out, int N, const int64_t *n, int64_t nrhs,
                                  const double *const *A, int prec, double rtol, int max_refine,
                                  int device, const sylv_tuning *tuning) {
    if (out) *out = nullptr;
    if (!A) return SYLV_ERR_INVALID_ARG;
    return create_plan(out, N, n, nrhs, nullptr, nullptr, nullptr, A, prec, rtol, max_refine,
                       device, tuning);
}

sylv_status sylv_plan_destroy(sylv_plan_t plan) {
    if (!plan) return SYLV_ERR_INVALID_ARG;
    batch_forget(plan);
    delete plan;
    return SYLV_OK;
}

sylv_status sylv_workspace_size(sylv_plan_t plan, size_t *bytes) {
    if (!plan || !bytes) return SYLV_ERR_INVALID_ARG;
    *bytes = plan->ws_bytes;
    return SYLV_OK;
}

sylv_status sylv_solve(sylv_plan_t p, const void *B, void *X, void *ws, size_t ws_bytes,
                       void *stream, sylv_info *info) {
    if (!p || !B || !X) return SYLV_ERR_INVALID_ARG;
    if (!p->fp64() && B == X) return SYLV_ERR_INVALID_ARG;
    if ((((uintptr_t)B) | ((uintptr_t)X)) & 15) return SYLV_ERR_INVALID_ARG;
    sylv_status s = check_ws(p, ws, ws_bytes);
    if (s != SYLV_OK) return s;
    DeviceGuard dg(p->device);
    if (!dg.ok) return SYLV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int launches = 0;
    s = solve_impl(p, B, X, ws, st, launches);
    if (s != SYLV_OK) return s;
    if (info) return fill_info(p, reinterpret_cast<DevFlags *>(ws), st, info, launches);
    return SYLV_OK;
}

sylv_status sylv_workspace_size_batched(int count, const sylv_plan_t *plans, size_t *bytes) {
    if (count < 0 || (count > 0 && !plans) || !bytes) return SYLV_ERR_INVALID_ARG;
    size_t tot = 0;
    for (int e = 0; e < count; ++e) {
        if (!plans[e]) return SYLV_ERR_INVALID_ARG;
        tot += align256(plans[e]->ws_bytes);
    }
    *bytes = tot;
    return SYLV_OK;
}

sylv_status sylv_solve_batched(int count, const sylv_plan_t *plans, const void *const *B,
                               void *const *X, void *ws, size_t ws_bytes, void *stream,
                               sylv_info *infos) {
    if (count < 0 || (count > 0 && (!plans || !B || !X))) return SYLV_ERR_INVALID_ARG;
    size_t need = 0;
    sylv_status s = sylv_workspace_size_batched(count, plans, &need);
    if (s != SYLV_OK) return s;
    if (need > 0 && (!ws || ws_bytes < need)) return SYLV_ERR_WORKSPACE;
    if (((uintptr_t)ws) & 255) return SYLV_ERR_INVALID_ARG;
    if (count == 0) return SYLV_OK;
    cudaStream_t st = (cudaStream_t)stream;
    bool direct = false;
    const int dev = plans[0]->device;
    for (int e = 0; e < count; ++e) {
        sylv_plan_s *p = plans[e];
        if (!B[e] || !X[e] || (!p->fp64() && B[e] == X[e])) return SYLV_ERR_INVALID_ARG;
        if ((((uintptr_t)B[e]) | ((uintptr_t)X[e])) & 15) return SYLV_ERR_INVALID_ARG;
        if (p->timing) direct = true;
        if (p->device != dev) return SYLV_ERR_INVALID_ARG;
    }
    DeviceGuard dg(dev);
    if (!dg.ok) return SYLV_ERR_CUDA;
    std::vector<int> launches((size_t)count, 0);
    if (direct) {
        size_t off = 0;
        for (int e = 0; e < count; ++e) {
            s = solve_impl(plans[e], B[e], X[e], (char *)ws + off, st, launches[(size_t)e]);
            if (s != SYLV_OK) return s;
            off += align256(plans[e]->ws_bytes);
        }
    } else {
        s = batch_graph_launch(count, plans, B, X, ws, st, launches);
        if (s != SYLV_OK) return s;
    }
    if (infos) {
        size_t off = 0;
        sylv_status worst = SYLV_OK;
        for (int e = 0; e < count; ++e) {
            sylv_status r = fill_info(plans[e], reinterpret_cast<DevFlags *>((char *)ws + off),
                                      st, &infos[e], launches[(size_t)e]);
            if (r != SYLV_OK && worst == SYLV_OK) worst = r;
            off += align256(plans[e]->ws_bytes);
        }
        return worst;
    }
    return SYLV_OK;
}

sylv_status sylv_plan_autotune(sylv_plan_t p, void *Tdev, void *ws, size_t ws_bytes,
                               void *stream, int32_t *block_out, float *best_ms) {
    if (!p || !Tdev) return SYLV_ERR_INVALID_ARG;
    sylv_status s = check_ws(p, ws, ws_bytes);
    if (s != SYLV_OK) return s;
    DeviceGuard dg(p->device);
    if (!dg.ok) return SYLV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t esz = p->fp64() ? p->ehi() : p->elo();
    batch_forget(p);
    if (cudaMemsetAsync(Tdev, 0, (size_t)(p->ntot * p->nrhs) * esz, st) != cudaSuccess)
        return SYLV_ERR_CUDA;
    Ctx c{p, st, reinterpret_cast<DevFlags *>(ws),
          reinterpret_cast<int *>((char *)ws + p->off_cnt)};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return SYLV_ERR_CUDA;
    auto time_cfg = [&](const SweepConfig &cfg, float &ms) -> bool {
        float best = 1e30f;
        int reps = 3;                                 // first run warms up
        for (int rep = 0; rep < reps; ++rep) {
            if (launch_solve_init(c.flags, st) != cudaSuccess) return false;
            if (cudaEventRecord(e0, st) != cudaSuccess) return false;
            if ((p->diag_sweep ? run_sweep(c, Tdev, p->fp64())
                               : run_sweep_cfg(c, cfg, Tdev, p->fp64())) != cudaSuccess)
                return false;
            if (cudaEventRecord(e1, st) != cudaSuccess) return false;
            if (cudaEventSynchronize(e1) != cudaSuccess) return false;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) best = std::min(best, t);
            if (rep == 0 && t > 10.f) reps = 2;       // long sweeps: one timed run
        }
        ms = best;
        return true;
    };
    float cur_ms = 0.f;
    bool ok = time_cfg(p->sweep, cur_ms);
    // the entrywise-division sweep (Remark 1) has no tiling to tune
    for (int target = 64; ok && !p->diag_sweep && target <= 2048; target *= 2) {
        int b[MAXM];
        choose_blocks(*p, target, nullptr, b);
        if (tiles_for(*p, b) > p->cnt_capacity) continue;
        for (int cand_i = 0; ok && cand_i < (p->fp64() ? 2 : 4); ++cand_i) {
            const int threads = (cand_i & 1) ? 256 : 128;
            const int sub = p->fp64() ? 1 : ((cand_i & 2) ? 4 : 1);
            // CTAs per SM: as many as fit, half of that, and 2 (fewer CTAs
            // shorten each tile's latency on the dependency chain)
            int pers[3] = {0, -1, -1};
            for (int pi = 0; ok && pi < 3; ++pi) {
                const int per = pers[pi];
                if (per < 0) continue;
                SweepConfig cand;
                if (build_sweep(*p, b, threads, cand, per, sub) != SYLV_OK) {
                    if (cand.dbuf) cudaFree(cand.dbuf);
                    break;
                }
                if (pi == 0) {
                    const int mx = cand.per_sm;
                    if (mx / 2 >= 2 && mx / 2 < mx) pers[1] = mx / 2;
                    if (mx > 2 && pers[1] != 2) pers[2] = 2;
                }
                float ms = 0.f;
                if (!time_cfg(cand, ms)) {
                    ok = false;
                    cudaFree(cand.dbuf);
                    break;
                }
                if (ms < cur_ms) {
                    cudaFree(p->sweep.dbuf);
                    p->sweep = cand;
                    cur_ms = ms;
                } else {
                    cudaFree(cand.dbuf);
                }
            }
        }
    }
    // transform passes: the plan's tensor-core passes with or without the TMA
    // pipeline, or CUDA-core passes only, at several fusion widths of adjacent
    // modes; each candidate times one forward and one back transform in place
    // on the scratch tensor
    if (ok && p->Nm > 0) {
        const int k = p->fp64() ? p->khi() : p->klo();
        auto time_tf = [&](float &ms) -> bool {
            float best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                if (cudaEventRecord(e0, st) != cudaSuccess) return false;
                if (run_groups(c, p->tgroups, p->fp64(), 0, Tdev, k, Tdev, k, Tdev, k, EPI_STORE,
                               nullptr) != cudaSuccess ||
                    run_groups(c, p->tgroups, p->fp64(), 1, Tdev, k, Tdev, k, Tdev, k, EPI_STORE,
                               nullptr) != cudaSuccess)
                    return false;
                if (cudaEventRecord(e1, st) != cudaSuccess) return false;
                if (cudaEventSynchronize(e1) != cudaSuccess) return false;
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) best = std::min(best, t);
            }
            ms = best;
            return true;
        };
        const std::vector<Group> orig = p->tgroups;
        const bool orig_plain = p->tc_plain;
        const int orig_gmax = p->tgroup_max;
        bool has_tc = false;
        for (const auto &g : orig) has_tc |= g.tc != 0;
        float best_ms = 1e30f;
        std::vector<Group> best_g = orig;
        bool best_plain = orig_plain;
        int best_gmax = orig_gmax;
        auto try_cand = [&](const std::vector<Group> &g, bool plain, int gm) {
            p->tgroups = g;
            p->tc_plain = plain;
            float ms = 0.f;
            if (!time_tf(ms)) { ok = false; return; }
            if (ms < best_ms) { best_ms = ms; best_g = g; best_plain = plain; best_gmax = gm; }
        };
        try_cand(orig, orig_plain, orig_gmax);
        if (ok && has_tc) try_cand(orig, !orig_plain, orig_gmax);
        for (int gm : {0, 64, 256, 1024, 4096}) {
            if (!ok) break;
            std::vector<Group> g;
            if (make_groups(*p, p->fp64(), true, gm, false, g) != SYLV_OK) continue;
            try_cand(g, orig_plain, gm);
        }
        p->tgroups = ok ? best_g : orig;
        p->tc_plain = ok ? best_plain : orig_plain;
        p->tgroup_max = ok ? best_gmax : orig_gmax;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return SYLV_ERR_CUDA;
    if (block_out)
        for (int j = 0, q = 0; j < p->N_in; ++j)
            block_out[j] = (q < p->Nm && p->orig[q] == j) ? p->sweep.a.b[q++] : 1;
    if (best_ms) *best_ms = cur_ms;
    return SYLV_OK;
}

// ------------------------------------------------------------ Theorem 1 --

sylv_status sylv_evolve_workspace_size(sylv_plan_t p, size_t *bytes) {
    if (!p || !bytes || p->real) return SYLV_ERR_INVALID_ARG;
    *bytes = align256(p->ws_bytes) + align256((size_t)(p->ntot * p->nrhs) * 16);
    return SYLV_OK;
}

sylv_status sylv_evolve(sylv_plan_t p, double t, const void *B, const void *X0, void *X,
                        void *ws, size_t ws_bytes, void *stream, sylv_info *info) {
    if (!p || !B || !X0 || !X || !std::isfinite(t) || p->real) return SYLV_ERR_INVALID_ARG;
    if ((((uintptr_t)B) | ((uintptr_t)X0) | ((uintptr_t)X)) & 15) return SYLV_ERR_INVALID_ARG;
    size_t need = 0;
    sylv_evolve_workspace_size(p, &need);
    if (!ws || ws_bytes < need) return SYLV_ERR_WORKSPACE;
    if (((uintptr_t)ws) & 255) return SYLV_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return SYLV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // exp(t A_j) on the host (Pade scaling and squaring), uploaded in stream order
    if (!p->evolve_ready || p->evolve_t != t) {
        // per mode: the complex entries, then the plane re + im
        size_t tot = 0;
        for (int j = 0; j < p->Nm; ++j) tot += (size_t)(3 * p->n[j] * p->n[j]);
        p->Ehost.assign(tot, 0.0);
        size_t o = 0;
        for (int j = 0; j < p->Nm; ++j) {
            const int64_t nj = p->n[j];
            const auto &Aj = p->Ah[p->orig[j]];
            std::vector<double> tA((size_t)(2 * nj * nj));
            for (size_t k = 0; k < (size_t)(nj * nj); ++k) {
                tA[2 * k] = t * Aj[k].real();
                tA[2 * k + 1] = t * Aj[k].imag();
            }
            double *Ej = p->Ehost.data() + o;
            sylv_status s = expm_host(nj, tA.data(), Ej);
            if (s != SYLV_OK) return s;
            for (size_t k = 0; k < (size_t)(nj * nj); ++k)
                Ej[2 * nj * nj + k] = Ej[2 * k] + Ej[2 * k + 1];
            o += (size_t)(3 * nj * nj);
        }
        o = 0;
        for (int j = 0; j < p->Nm; ++j) {
            const size_t bytes = (size_t)(p->n[j] * p->n[j]) * 24;
            if (cudaMemcpyAsync(const_cast<void *>(p->E64[j]), p->Ehost.data() + o, bytes,
                                cudaMemcpyHostToDevice, st) != cudaSuccess)
                return SYLV_ERR_CUDA;
            o += bytes / 8;
        }
        p->evolve_eps = std::exp(t * p->sigma);
        if (!std::isfinite(p->evolve_eps.real()) || !std::isfinite(p->evolve_eps.imag()))
            return SYLV_ERR_INVALID_ARG;
        if (p->oz) {
            // digits of exp(t A_j) for the tensor-core passes (exp(t sigma) folded
            // into the first mode)
            size_t total = 0;
            for (auto &o : p->ozpasses) total += (size_t)6 * o.aimg_bytes;
            p->Eimg_host.assign(total, 0);
            size_t off = 0;
            for (auto &o : p->ozpasses) {
                const int64_t nj = o.n;
                std::vector<cd> Em((size_t)(nj * nj));
                size_t base = 0;
                for (int q = 0; q < o.j; ++q) base += (size_t)(3 * p->n[q] * p->n[q]);
                for (size_t k = 0; k < Em.size(); ++k)
                    Em[k] = cd(p->Ehost[base + 2 * k], p->Ehost[base + 2 * k + 1]) *
                            (o.j == 0 ? p->evolve_eps : cd(1.0));
                o.eE = digit_images(Em, o, p->Eimg_host.data() + off);
                if (cudaMemcpyAsync(const_cast<unsigned char *>(o.eimg), p->Eimg_host.data() + off,
                                    (size_t)6 * o.aimg_bytes, cudaMemcpyHostToDevice, st) !=
                    cudaSuccess)
                    return SYLV_ERR_CUDA;
                off += (size_t)6 * o.aimg_bytes;
            }
        }
        p->evolve_t = t;
        p->evolve_ready = true;
    }
    Ctx c{p, st, reinterpret_cast<DevFlags *>(ws),
          reinterpret_cast<int *>((char *)ws + p->off_cnt)};
    void *W = (char *)ws + align256(p->ws_bytes);
    phase_begin(c, SYLV_PH_EVOLVE);
    if (launch_solve_init(c.flags, st) != cudaSuccess) return SYLV_ERR_CUDA;
    count(c);
    if (p->oz) {
        // the same two steps as digit products on the tensor cores: W = B + sum_j
        // A_j (x)_j X0 (sigma in the first mode's digits), then F = E_N (x)_N ( ...
        // E_1 (x)_1 W) - B one mode at a time, in place on W
        const int64_t cnt = p->ntot * p->nrhs;
        void *Rdf = (char *)ws + p->off_R;
        const size_t np = p->ozpasses.size();
        if (launch_maxabs(X0, cnt, c.flags, p->num_sms, st) != cudaSuccess) return SYLV_ERR_CUDA;
        count(c);
        for (size_t k = 0; k < np; ++k) {
            const auto &o = p->ozpasses[k];
            if (run_oz_pass(c, k, o.aimg, o.eA, X0, B, Rdf, Rdf, W,
                            k == 0 ? OZ_IN_B : OZ_IN_PAIRS,
                            k + 1 == np ? OZ_OUT_C128 : OZ_OUT_PAIRS, 1, 1.f, nullptr) != cudaSuccess)
                return SYLV_ERR_CUDA;
        }
        for (size_t k = 0; k < np; ++k) {
            const auto &o = p->ozpasses[k];
            if (launch_maxabs(W, cnt, c.flags, p->num_sms, st) != cudaSuccess)
                return SYLV_ERR_CUDA;
            count(c);
            if (run_oz_pass(c, k, o.eimg, o.eE, W, B, nullptr, nullptr, W,
                            k + 1 == np ? OZ_IN_B : OZ_IN_ZERO, OZ_OUT_C128, 1, -1.f,
                            nullptr) != cudaSuccess)
                return SYLV_ERR_CUDA;
        }
    } else {
        // W = B + sigma X0 + sum_j A_j (x)_j X0  (residual passes with -A_j, -sigma)
        const cd nsig = -p->sigma;
        if (run_residual(c, B, X0, W, nullptr, p->nA64, &nsig) != cudaSuccess)
            return SYLV_ERR_CUDA;
        // F = exp(t sigma) exp(t A_N) (x)_N ( ... exp(t A_1) (x)_1 W) - B, Eq. (C)
        if (run_groups(c, p->egroups, true, 0, W, ELEM_C128, W, ELEM_C128, W, ELEM_C128, EPI_SUB,
                       nullptr, p->E64, B, p->evolve_eps) != cudaSuccess)
            return SYLV_ERR_CUDA;
    }
    phase_end(c);
    // sum_j A_j (x)_j X(t) = F, Eq. (sylvesterNDC)
    int launches = 0;
    sylv_status s = solve_impl(p, W, X, ws, st, launches);
    if (s != SYLV_OK) return s;
    if (cudaGetLastError() != cudaSuccess) return SYLV_ERR_CUDA;
    if (info) return fill_info(p, c.flags, st, info, c.launches + launches);
    return SYLV_OK;
}

sylv_status sylv_forward(sylv_plan_t p, void *Tdev, void *ws, size_t ws_bytes, void *stream) {
    if (!p || !Tdev) return SYLV_ERR_INVALID_ARG;
    sylv_status s = check_ws(p, ws, ws_bytes);
    if (s != SYLV_OK) return s;
    DeviceGuard dg(p->device);
    if (!dg.ok) return SYLV_ERR_CUDA;
    Ctx c{p, (cudaStream_t)stream, reinterpret_cast<DevFlags *>(ws), nullptr};
    if (p->Nm == 0) return SYLV_OK;
    int k = p->fp64() ? p->khi() : p->klo();
    if (run_groups(c, p->tgroups, p->fp64(), 0, Tdev, k, Tdev, k, Tdev, k, EPI_STORE, nullptr) !=
        cudaSuccess)
        return SYLV_ERR_CUDA;
    return SYLV_OK;
}

sylv_status sylv_back(sylv_plan_t p, void *Tdev, void *ws, size_t ws_bytes, void *stream) {
    if (!p || !Tdev) return SYLV_ERR_INVALID_ARG;
    sylv_status s = check_ws(p, ws, ws_bytes);
    if (s != SYLV_OK) return s;
    DeviceGuard dg(p->device);
    if (!dg.ok) return SYLV_ERR_CUDA;
    Ctx c{p, (cudaStream_t)stream, reinterpret_cast<DevFlags *>(ws), nullptr};
    if (p->Nm == 0) return SYLV_OK;
    int k = p->fp64() ? p->khi() : p->klo();
    if (run_groups(c, p->tgroups, p->fp64(), 1, Tdev, k, Tdev, k, Tdev, k, EPI_STORE, nullptr) !=
        cudaSuccess)
        return SYLV_ERR_CUDA;
    return SYLV_OK;
}

sylv_status sylv_sweep(sylv_plan_t p, void *Tdev, void *ws, size_t ws_bytes, void *stream) {
    if (!p || !Tdev) return SYLV_ERR_INVALID_ARG;
    sylv_status s = check_ws(p, ws, ws_bytes);
    if (s != SYLV_OK) return s;
    DeviceGuard dg(p->device);
    if (!dg.ok) return SYLV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    Ctx c{p, st, reinterpret_cast<DevFlags *>(ws),
          reinterpret_cast<int *>((char *)ws + p->off_cnt)};
    if (launch_solve_init(c.flags, st) != cudaSuccess) return SYLV_ERR_CUDA;
    if (run_sweep(c, Tdev, p->fp64()) != cudaSuccess) return SYLV_ERR_CUDA;
    return SYLV_OK;
}

sylv_status sylv_residual(sylv_plan_t p, const void *B, const void *X, void *R, void *stream) {
    if (!p || !B || !X || !R || R == B || R == X) return SYLV_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (!dg.ok) return SYLV_ERR_CUDA;
    Ctx c{p, (cudaStream_t)stream, nullptr, nullptr};
    if (run_residual(c, B, X, R, nullptr) != cudaSuccess) return SYLV_ERR_CUDA;
    return SYLV_OK;
}

sylv_status sylv_plan_factors(sylv_plan_t p, int j, double *Qo, double *To) {
    if (!p || !Qo || !To || j < 0 || j >= p->N_in) return SYLV_ERR_INVALID_ARG;
    if (p->real) {            // real Q_j and quasi-triangular T_j, zero imaginary parts
        const auto &Q = p->Qr[(size_t)j];
        const auto &T = p->Tr[(size_t)j];
        for (size_t k = 0; k < Q.size(); ++k) {
            Qo[2 * k] = Q[k]; Qo[2 * k + 1] = 0.0;
            To[2 * k] = T[k]; To[2 * k + 1] = 0.0;
        }
        return SYLV_OK;
    }
    const auto &Q = p->Qh[(size_t)j];
    const auto &T = p->Th[(size_t)j];
    for (size_t k = 0; k < Q.size(); ++k) {
        Qo[2 * k] = Q[k].real(); Qo[2 * k + 1] = Q[k].imag();
        To[2 * k] = T[k].real(); To[2 * k + 1] = T[k].imag();
    }
    return SYLV_OK;
}

sylv_status sylv_plan_describe(sylv_plan_t p, sylv_plan_desc *out) {
    if (!p || !out) return SYLV_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->transform_passes = p->Nm > 0 ? (int32_t)p->tgroups.size() : 0;
    for (const auto &g : p->tgroups) out->transform_tc_passes += g.tc ? 1 : 0;
    if (!p->fp64()) {
        out->residual_tc = p->oz ? 1 : 0;
        out->residual_passes = p->oz ? (int32_t)p->ozpasses.size() : (int32_t)p->rgroups.size();
    }
    out->diag_sweep = p->diag_sweep ? 1 : 0;
    const SweepArgs &a = p->sweep.a;
    out->sweep_threads = p->sweep.threads;
    out->sweep_ctas_per_sm = p->sweep.per_sm;
    out->sweep_grid = p->sweep.grid;
    out->sweep_tiles = a.ntiles;
    out->sweep_tile_entries = a.Pt;
    int lev = 1;
    for (int j = 0; j < p->Nm; ++j) lev += a.Bc[j] - 1;
    out->sweep_tile_levels = lev;
    out->sweep_inv_table = p->inv_tab ? 1 : 0;
    out->sweep_far_split = a.far_split;
    for (int j = 0, q = 0; j < p->N_in && j < 64; ++j)
        out->sweep_block[j] = (q < p->Nm && p->orig[q] == j) ? a.b[q++] : 1;
    out->sweep_lanes = a.fast ? a.sub : 1;
    out->transform_tma = 0;
    for (const auto &g : p->tgroups)
        if (g.tc && !g.mode1 && !p->tc_plain && g.L % 64 == 0 && g.P <= 64 && !g.cview)
            out->transform_tma += 1;
    out->transform_group_max = p->tgroup_max;
    out->sweep_3m = a.g3;
    out->transform_fib_passes = 0;
    for (const auto &g : p->tgroups) out->transform_fib_passes += g.fib ? 1 : 0;
    return SYLV_OK;
}

sylv_status sylv_plan_set_timing(sylv_plan_t p, int enable) {
    if (!p) return SYLV_ERR_INVALID_ARG;
    p->timing = enable != 0;
    return SYLV_OK;
}

sylv_status sylv_plan_timing(sylv_plan_t p, sylv_timing *out, int reset) {
    if (!p || !out) return SYLV_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    std::memset(out, 0, sizeof(*out));
    for (auto &ph : p->tphases) {
        if (cudaEventSynchronize(ph.b) != cudaSuccess) return SYLV_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ph.a, ph.b) != cudaSuccess) return SYLV_ERR_CUDA;
        out->ms[ph.phase] += ms;
        out->launches[ph.phase] += ph.launches;
    }
    out->solves = p->timed_solves;
    if (reset) {
        for (auto &ph : p->tphases) {
            p->ev_free.push_back(ph.a);
            p->ev_free.push_back(ph.b);
        }
        p->tphases.clear();
        p->timed_solves = 0;
    }
    return SYLV_OK;
}

}  // extern "C"

// ======================================================= scratch-free sweep ==
// sylv_sweep_static serves callers that cannot allocate device memory (a fixed
// budget already reserved by another allocator, or a loop where an allocation
// would stall on a device synchronisation).  Its scratch is this array: one
// per device that loads the library, held until the process exits.  Host code
// must not hand `g_static_scratch` itself to a kernel (on the host it names a
// host-side stand-in); the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[SYLV_STATIC_SCRATCH_BYTES];

namespace {
constexpr int STATIC_MAX_DEVICES = 64;
std::mutex g_static_mu;
void *g_static_addr[STATIC_MAX_DEVICES] = {};

// Device address of the array on `dev` (which must be current); looked up
// once per device, on the first call there.
sylv_status static_scratch(int dev, void **out) {
    if (dev < 0 || dev >= STATIC_MAX_DEVICES) return SYLV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return SYLV_ERR_CUDA;
        }
        g_static_addr[dev] = ptr;
    }
    *out = g_static_addr[dev];
    return SYLV_OK;
}
}  // namespace

extern "C" sylv_status sylv_sweep_static(sylv_plan_t p, void *Tdev, void *stream) {
    if (!p || !Tdev) return SYLV_ERR_INVALID_ARG;
    const size_t cnt_off = align256(sizeof(DevFlags));
    // the entrywise-division sweep (Remark 1) uses the control block only; the
    // tiled sweep also one int counter per tile
    if (!p->diag_sweep &&
        cnt_off + align256((size_t)p->sweep.a.ntiles * 4) > SYLV_STATIC_SCRATCH_BYTES)
        return SYLV_ERR_SHAPE;
    DeviceGuard dg(p->device);
    if (!dg.ok) return SYLV_ERR_CUDA;
    void *base = nullptr;
    sylv_status s = static_scratch(p->device, &base);
    if (s != SYLV_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Ctx c{p, st, reinterpret_cast<DevFlags *>(base),
          reinterpret_cast<int *>((char *)base + cnt_off)};
    // the array keeps the previous call's control block: clear it (done, err,
    // ticket); run_sweep then rewrites every tile counter before the sweep
    if (launch_solve_init(c.flags, st) != cudaSuccess) return SYLV_ERR_CUDA;
    if (run_sweep(c, Tdev, p->fp64()) != cudaSuccess) return SYLV_ERR_CUDA;
    return SYLV_OK;
}

// Host side of libqmc_gb300: argument validation against the paper's
// definitions, the block schedule (Algorithm 2's weight blocks split into a
// register-tree fine band and coarse block products), the workspace layout,
// and the launch sequences behind the C ABI of include/qmc.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/qmc.h"
#include "qmc_internal.cuh"

using namespace qmc;

namespace {

thread_local std::string g_err;

qmc_status fail(qmc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define QMC_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(QMC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ------------------------------------------------------------------------------------------
// kernel tracing: while enabled, every launch is bracketed by CUDA events on its stream
// ------------------------------------------------------------------------------------------
struct TraceRec {
    const char* name;
    cudaEvent_t a, b;
};
struct TraceState {
    std::mutex mu;
    bool on = false;
    std::vector<TraceRec> recs;
    std::vector<cudaEvent_t> pool;
    std::vector<std::string> names;
    std::vector<unsigned long long> counts;
    std::vector<double> ms;
};
TraceState& trace_state() {
    static TraceState t;
    return t;
}
cudaEvent_t trace_event(TraceState& t) {
    if (!t.pool.empty()) {
        cudaEvent_t e = t.pool.back();
        t.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
struct TraceScope {
    cudaStream_t st;
    const char* name;
    cudaEvent_t a = nullptr, b = nullptr;
    bool on = false;
    TraceScope(cudaStream_t s, const char* n) : st(s), name(n) {
        TraceState& t = trace_state();
        std::lock_guard<std::mutex> g(t.mu);
        if (!t.on) return;
        on = true;
        a = trace_event(t);
        b = trace_event(t);
        cudaEventRecord(a, st);
    }
    ~TraceScope() {
        if (!on) return;
        cudaEventRecord(b, st);
        TraceState& t = trace_state();
        std::lock_guard<std::mutex> g(t.mu);
        t.recs.push_back({name, a, b});
    }
};
#define QMC_LAUNCH(st, name, call)        \
    do {                                  \
        TraceScope ts_((st), (name));     \
        QMC_CUDA(call);                   \
    } while (0)

// GF(2) rank of n vectors of at most 32 bits: each vector is reduced against an XOR basis indexed
// by leading bit and joins it if something is left (no allocation: the check runs on every call)
int gf2_rank(const uint32_t* v, int n) {
    uint32_t basis[32] = {0};
    int rank = 0;
    for (int i = 0; i < n; ++i) {
        uint32_t x = v[i];
        while (x) {
            const int b = 31 - __builtin_clz(x);
            if (!basis[b]) {
                basis[b] = x;
                ++rank;
                break;
            }
            x ^= basis[b];
        }
    }
    return rank;
}

qmc_status validate(const qmc_rule* r) {
    if (!r) return fail(QMC_ERR_INVALID_ARG, "rule is NULL");
    if (r->kind != QMC_LATTICE && r->kind != QMC_DIGITAL_NET && r->kind != QMC_REDUCED_MC &&
        r->kind != QMC_POLY_LATTICE)
        return fail(QMC_ERR_INVALID_ARG, "kind %d is not QMC_LATTICE, QMC_DIGITAL_NET, QMC_REDUCED_MC or "
                    "QMC_POLY_LATTICE", r->kind);
    if (r->b < 2) return fail(QMC_ERR_INVALID_ARG, "base b=%u must be a prime >= 2", r->b);
    for (uint32_t d = 2; d * d <= r->b; ++d)
        if (r->b % d == 0) return fail(QMC_ERR_INVALID_ARG, "base b=%u is not prime", r->b);
    if (r->m < 1) return fail(QMC_ERR_INVALID_ARG, "m=%u: N = b^m needs m >= 1", r->m);
    if (r->b == 2 && r->m > 30) return fail(QMC_ERR_UNSUPPORTED, "m=%u: N = 2^m is limited to m <= 30", r->m);
    if (r->b > 2) {
        // Sec. 1.3 lattices and Sec. 5 reduced MC in base b; nets and polynomial lattices over F_b are
        // not built
        if (r->kind != QMC_LATTICE && r->kind != QMC_REDUCED_MC)
            return fail(QMC_ERR_UNSUPPORTED, "base b=%u: only lattices and reduced Monte Carlo are built", r->b);
        unsigned long long N = 1;
        for (uint32_t i = 0; i < r->m; ++i) {
            N *= r->b;
            if (N > (1ull << 31)) return fail(QMC_ERR_UNSUPPORTED, "N = %u^%u exceeds 2^31 points", r->b, r->m);
        }
    }
    if (r->s < 1 || r->s > 65536) return fail(QMC_ERR_INVALID_ARG, "s=%u outside [1, 65536]", r->s);
    if (!r->w) return fail(QMC_ERR_INVALID_ARG, "w is NULL");
    for (uint32_t j = 1; j < r->s; ++j)
        if (r->w[j] < r->w[j - 1])
            return fail(QMC_ERR_INVALID_ARG, "w must be nondecreasing: w[%u]=%u < w[%u]=%u", j, r->w[j], j - 1,
                        r->w[j - 1]);
    if (r->transform < QMC_T_IDENTITY || r->transform > QMC_T_TENT)
        return fail(QMC_ERR_INVALID_ARG, "transform %d unknown", r->transform);
    if (r->R > 65535) return fail(QMC_ERR_INVALID_ARG, "R=%u shifts: at most 65535", r->R);
    const uint32_t m = r->m;
    // b^e for the base's exponents (b^m <= 2^31 for b > 2 was checked above)
    auto bpow = [&](uint32_t e) -> unsigned long long {
        unsigned long long v = 1;
        for (uint32_t i = 0; i < e; ++i) v *= r->b;
        return v;
    };
    if (r->kind == QMC_REDUCED_MC) {
        // Sec. 5: the caller's i.i.d. samples, N_j = b^(m - min(w_j, m)) per column and replica
        if (!r->z) return fail(QMC_ERR_INVALID_ARG, "reduced MC needs its samples in z");
        if (r->C || r->shift || r->d_shift)
            return fail(QMC_ERR_INVALID_ARG, "reduced MC takes no C and no shift (R counts independent replicas)");
        if (r->transform == QMC_T_INV_NORMAL) {
            unsigned long long T = 0;
            for (uint32_t j = 0; j < r->s; ++j) T += bpow(m - std::min(r->w[j], m));
            // (blocks reduced by a branch-free minimum, which the compiler vectorises; a block
            // holding a zero is then searched for its index)
            const unsigned long long words = T * std::max<uint32_t>(r->R, 1);
            const uint32_t* zw = r->z;
            for (unsigned long long i0 = 0; i0 < words; i0 += 4096) {
                const unsigned long long i1 = std::min(words, i0 + 4096);
                uint32_t mn = 0xFFFFFFFFu;
                for (unsigned long long i = i0; i < i1; ++i) mn = std::min(mn, zw[i]);
                if (mn != 0) continue;
                for (unsigned long long i = i0; i < i1; ++i)
                    if (zw[i] == 0)
                        return fail(QMC_ERR_INVALID_ARG,
                                    "sample word %llu is 0: the inverse-normal transform maps it to -inf", i);
            }
        }
        return QMC_OK;
    }
    if (r->R > 0 && !r->shift) return fail(QMC_ERR_INVALID_ARG, "R=%u but shift is NULL", r->R);
    if (r->transform == QMC_T_INV_NORMAL && r->R == 0)
        return fail(QMC_ERR_INVALID_ARG, "the inverse-normal transform needs a random shift (x=0 maps to -inf)");
    if (r->b > 2) {
        // z_j in U_{b^q}: 1 <= z_j < b^q and not divisible by the prime b (z_j = 1 when q = 0)
        if (!r->z) return fail(QMC_ERR_INVALID_ARG, "lattice rule needs z");
        for (uint32_t j = 0; j < r->s; ++j) {
            const uint32_t q = m - std::min(r->w[j], m);
            const unsigned long long n = bpow(q);
            const uint32_t z = r->z[j];
            if (q == 0 ? z != 1 : (z < 1 || z % r->b == 0 || z >= n))
                return fail(QMC_ERR_INVALID_ARG, "z[%u]=%u not in U_{%u^%u}", j, z, r->b, q);
        }
        if (r->transform == QMC_T_INV_NORMAL) {
            // the shifted point {u / b^q + D 2^-32} is formed in double: reject a shift that puts a point
            // within 2^-50 of 1 (the rounded sum could reach 1, so the point 0 and -inf), or D = 0 (the
            // point u = 0 stays 0).  The nearest u / b^q to 1 - D 2^-32 is found in exact integers.
            for (uint32_t i = 0; i < r->R; ++i)
                for (uint32_t j = 0; j < r->s; ++j) {
                    const unsigned long long D = r->shift[(size_t)i * r->s + j];
                    const uint32_t q = m - std::min(r->w[j], m);
                    const long long n = (long long)bpow(q);
                    const long long e = (long long)((1ull << 32) - D);          // 2^32 (1 - D 2^-32)
                    bool near = D == 0;
                    const long long u0 = (long long)(((unsigned long long)e * (unsigned long long)n) >> 32);
                    for (long long u = u0 - 1; u <= u0 + 1 && !near; ++u) {
                        if (u < 0 || u >= n) continue;
                        const long long diff = u * (1LL << 32) - e * n;          // 2^32 n (u/n - (1 - D 2^-32))
                        const unsigned long long ad = (unsigned long long)(diff < 0 ? -diff : diff);
                        if (ad < (unsigned long long)n && (ad << 18) < (unsigned long long)n) near = true;
                    }
                    if (near)
                        return fail(QMC_ERR_INVALID_ARG, "shift %u of column %u (0x%llx) puts a point at or within "
                                    "2^-50 of 0 under the inverse-normal transform", i, j, D);
                }
        }
        return QMC_OK;
    }
    if (r->transform == QMC_T_INV_NORMAL) {
        // Column j takes, over one period, every value u 2^(32-q) with u < 2^q (q = m - min(w_j, m)):
        // the lattice's u = k z_j mod 2^q with z_j odd, the polynomial lattice's carry-less product with
        // gt_j(0) = 1 and the net's nonsingular leading block are all bijections.  So the shifted column
        // reaches X32 = 0, which the inverse normal maps to -inf, exactly when the low 32 - q bits of
        // D_j vanish ((u 2^(32-q) + D_j) mod 2^32 = 0 and (u 2^(32-q)) XOR D_j = 0 each have a solution u).
        for (uint32_t i = 0; i < r->R; ++i)
            for (uint32_t j = 0; j < r->s; ++j) {
                const uint32_t q = m - std::min(r->w[j], m), low = 32 - q;
                const uint32_t mask = low >= 32 ? 0xFFFFFFFFu : ((1u << low) - 1u);
                if ((r->shift[(size_t)i * r->s + j] & mask) == 0)
                    return fail(QMC_ERR_INVALID_ARG,
                                "shift %u of column %u (0x%x) has its low %u bits zero: a shifted point is 0, which "
                                "the inverse-normal transform maps to -inf", i, j, r->shift[(size_t)i * r->s + j], low);
            }
    }
    if (r->kind == QMC_LATTICE || r->kind == QMC_POLY_LATTICE) {
        // z_j in U_{2^q}; for polynomials: gt_j(0) = 1 and deg gt_j < q (gcd(gt_j, x^q) = 1)
        const char* what = r->kind == QMC_LATTICE ? "lattice rule needs z" : "polynomial lattice rule needs z";
        if (!r->z) return fail(QMC_ERR_INVALID_ARG, "%s", what);
        for (uint32_t j = 0; j < r->s; ++j) {
            const uint32_t q = m - std::min(r->w[j], m);
            const uint32_t z = r->z[j];
            if (q == 0) {
                if (z != 1) return fail(QMC_ERR_INVALID_ARG, "z[%u]=%u: U_1 = {1} when w_j >= m", j, z);
            } else if (z < 1 || (z & 1u) == 0 || (uint64_t)z >= (1ull << q)) {
                return fail(QMC_ERR_INVALID_ARG, "z[%u]=%u not in U_{2^%u} (odd, < 2^%u)", j, z, q, q);
            }
        }
    } else {
        if (!r->C) return fail(QMC_ERR_INVALID_ARG, "digital net needs C");
        for (uint32_t j = 0; j < r->s; ++j) {
            const uint32_t wcl = std::min(r->w[j], m), q = m - wcl;
            const uint32_t rowmask = (wcl >= 32) ? 0u : ~((1u << wcl) - 1u);
            uint32_t rows[32];
            for (uint32_t c = 0; c < m; ++c) {
                const uint32_t word = r->C[(size_t)j * m + c];
                if (m < 32 && (word >> m) != 0)
                    return fail(QMC_ERR_INVALID_ARG, "C[%u][%u]=0x%x has bits above row 1 (bit m-1)", j, c, word);
                rows[c] = (word & rowmask) >> wcl;     // eq. reduced_genmat_net2: the first q rows remain
            }
            // The first q rows of the reduced C^(j) must be linearly independent over GF(2), so that
            // column j takes every value v 2^-q, v < 2^q, exactly 2^{w_j} times (Sec. 4).  For a periodic
            // net (columns q+1.. zero) this is the nonsingular leading block.
            if (gf2_rank(rows, (int)m) != (int)q)
                return fail(QMC_ERR_INVALID_ARG, "the first %u rows of the reduced C^(%u) have GF(2) rank below %u", q, j,
                            q);
        }
    }
    return QMC_OK;
}

// A net whose reduced matrices have a nonzero column beyond m - w_j (Sec. 4: reduced by rows, not
// periodic in the point index): Algorithm 4's case.
bool net_nonperiodic(const qmc_rule* r) {
    if (r->kind != QMC_DIGITAL_NET) return false;
    const uint32_t m = r->m;
    for (uint32_t j = 0; j < r->s; ++j) {
        const uint32_t wcl = std::min(r->w[j], m), q = m - wcl;
        const uint32_t rowmask = (wcl >= 32) ? 0u : ~((1u << wcl) - 1u);
        for (uint32_t c = q; c < m; ++c)
            if (r->C[(size_t)j * m + c] & rowmask) return true;
    }
    return false;
}

// ------------------------------------------------------------------------------------------
// schedule autotuning: per problem shape, the fine band's forward column groups (columns per
// CTA = 4 qpg) and adjoint roots per CTA, measured by qmc_autotune; 0 keeps the cost model's
// choice.  The planner consults the cache on every call; qmc_autotune passes its candidates
// through a thread-local hint.
// ------------------------------------------------------------------------------------------
struct TuneVal {
    int fwd_qpg = 0;
    int bwd_rpc = 0;
    int coarse = 0;                // tensor-core tiers: 1 level passes, 2 block products + chain sum
    int bwd = 0;                   // tensor-core adjoint: 1 one fold + k_coarse_grad_tc, 2 the fused
                                   // fold-gradient and TMA gradient kernels (0: by size)
    int fwd_nb = 0;                // S4 forward: level-3 nodes per thread, 1 or 2 (0: by integrand)
    int bwd_cpl = 0;               // S4 adjoint: column pairs per lane, 1 or 2 (0: 2)
};
struct TuneCache {
    std::mutex mu;
    std::map<std::string, TuneVal> m;
};
TuneCache& tune_cache() {
    static TuneCache c;
    return c;
}
thread_local const TuneVal* t_hint = nullptr;

// ------------------------------------------------------------------------------------------
// the plan: block schedule and workspace layout of one problem
// ------------------------------------------------------------------------------------------
struct Plan {
    int op = 0;
    int kind = 0, m = 0, s = 0, transform = 0, R = 0, reff = 1;
    long long N = 0;
    int lev_tau[kMaxLevels] = {}, lev_col0[kMaxLevels] = {};
    long long lev_tab[kMaxLevels + 1] = {};
    long long T_tot = 0, tab_stride = 0;   // table entries per shift, and the per-shift stride (multiple of 4)
    int tau = 0, tau_pad = 0, precision = 0, elt = 4, fkind = 0;
    int shape = SHAPE_S0, JF = 0, kf_width = 0, cw_bwd = 4;
    int fwd_nb = 1;                // S4 forward: level-3 nodes per thread
    int bwd_cpl = 1;               // S4 adjoint: column pairs per lane
    bool exact = false;            // fine band levels hold exactly their maximum column counts
    Chain chf{}, chb{};
    long long B_per_shift = 0, S_per_shift = 0, partc_elems = 0, Fchain_per_shift = 0;
    FoldLevels fold{};
    int root_blocks = 0, cg_count = 1, cr = 0;
    int groups = 0, roots_per_cta = 8, passes = 0, bwd_tiles = 0;
    // tensor-core backward: entries staged by TMA (k_grad_tc; whole chunks of 32 rows, F materialised)
    // and the rest on k_coarse_grad_tc (chl, its tiles bwd_tiles_l)
    int gsel[kMaxGradTc] = {}, ngsel = 0, bwd_tiles_l = 0;
    long long gxoff[kMaxGradTc] = {};   // their pre-split table columns in the split buffer
    bool bwd_tma = false;               // large enough for the fused and TMA gradient kernels
    bool froot_tiled = false;           // root gradients in 128-column tiles (the fused kernel reads them)
    Chain chl{};
    // tensor-core backward of the lowest fg_L coarse levels in one pass over the root gradients
    // (k_fold_grad_tc, entries fg_ent[d] of level JF + d or -1), the folds above JF + fg_L from
    // F_{JF+fg_L} (fold2), the levels' table columns pre-split at off_xt
    int fg_L = 0, fg_ent[kMaxFoldLv] = {-1, -1, -1};
    FoldGradArgs fga{};
    SplitXtArgs sxa{};
    FoldLevels fold2{};
    size_t off_xt = 0, xt_bytes = 0;
    int nblk = 0;
    int tc_pieces = 0;             // 3: split tier, 1: bf16 tier, 0: FP32 / FP64 block products
    bool fine_s4 = false;          // S4 band in FP32 on the CUDA cores (every float tier)
    bool fine_mat = false;         // materialised S4 band of the float tiers (column-pair lanes)
    bool need_gen = false, need_shift = false, need_pad = false;
    std::string tune_key;          // the problem shape the schedule cache is keyed by
    TuneVal tuned{};               // the cached (or hinted) schedule applied to this plan
    bool lv = false;               // tensor-core tiers: Algorithm 2 top down (k_level_tc passes)
    LevelPlan lvp{};
    bool has_shift = false;        // lattice / net with R shifts (reduced MC: R replicas, no shift)
    bool nonper = false;           // non-periodic reduced net: every column on level 0 with N rows
    // tensor-core tiers with points in [0, 1) (identity, tent): the block products take x - 1/2, so
    // that their terms take both signs (the tensor core's FP32 accumulation rounds toward zero, which
    // biases long sums of terms of one sign), and the constant 1/2 returns as one exact term
    float xc = 0.0f;
    size_t off_gsum = 0;           // backward: column sums of the folded gradient (65 x tau_pad doubles)
    // base b > 2: the levels with columns from the coarsest down, each written at bl_rows rows
    bool base_b = false;
    int b = 2;
    long long lev_n[kMaxLevels] = {};
    int bl_n = 0, bl_lev[kMaxLevels] = {};
    long long bl_rows[kMaxLevels] = {}, bl_kper[kMaxLevels] = {};
    int bl_split[kMaxLevels] = {};
    size_t bl_out[kMaxLevels] = {}, bl_F[kMaxLevels] = {}, bl_part[kMaxLevels] = {}, off_G = 0;
    size_t off_gen = 0, off_shift = 0, off_A = 0, off_tab = 0, off_B = 0, off_S = 0, off_rowpart = 0, off_rowmax = 0,
           off_rowsave = 0, off_fpart = 0, off_ticket = 0, off_F = 0, off_Fchain = 0, off_gradpart = 0, off_partc = 0,
           total = 0;
};

// words of the rule's generator: z (lattice), the column masks C (net), or the samples of every
// replica (reduced MC: R_eff x sum_j N_j, the distinct-row table's layout)
size_t gen_words(const Plan& P) {
    if (P.kind == QMC_DIGITAL_NET) return (size_t)P.s * P.m;
    if (P.kind == QMC_REDUCED_MC) return (size_t)P.reff * (size_t)P.T_tot;
    return (size_t)P.s;
}

// Algorithm 2 on the tensor cores (split and bf16 tiers): the coarse levels I >= JF with columns,
// from the top down, as passes of k_level_tc.  Levels with fewer than 128 distinct rows go
// together into the first passes (their rows are stored repeated up to a 128-row tile); every
// other level is a pass of its own, except that the two lowest levels share the last pass
// (which writes the root values S): that pass then multiplies the second level on twice its
// distinct rows, but the level's partial sum (half the size of S) is never written or read.
// Falls back to the block products and chain sum when a limit below is exceeded.
// columns of a root-gradient row as stored: tau_pad, or whole 128-column tiles when tiled
long long root_cols(const Plan& P) { return P.froot_tiled ? (long long)(P.tau_pad + 127) / 128 * 128 : P.tau_pad; }

void plan_levels(Plan& P) {
    LevelPlan& L = P.lvp;
    L = LevelPlan{};
    L.pieces = P.tc_pieces;
    const int t_tiles = (P.tau_pad + 255) / 256;
    L.tA = t_tiles * 256;
    int levs[kMaxLevels], nl = 0;
    for (int I = P.m; I >= P.JF; --I)
        if (P.lev_tau[I] > 0) levs[nl++] = I;
    if (nl == 0) return;
    // group: [tiny levels in groups of kMaxPassSeg] [one level each] ... [the two lowest]
    int group[kMaxLevels], ng = 0, i = 0;
    while (i < nl && P.m - levs[i] < 7) {
        int k = 0;
        while (i + k < nl && P.m - levs[i + k] < 7 && k < kMaxPassSeg) ++k;
        group[ng++] = k;
        i += k;
    }
    // The last pass writes S and is bound by that write; the lowest levels share it while their
    // block products, taken over all n_root rows there, stay well inside the write time (at most
    // 128 columns in the split tier's six piece products, 512 in the bf16 tier), at least two.
    // Each level moved in saves its partial sum's write and read-back.
    int k_last = 0;
    {
        const int kmax = P.tc_pieces == 3 ? 128 : 512;
        int cols = 0;
        for (int j = nl - 1; j >= i && k_last < kMaxPassSeg; --j) {
            if (k_last >= 2 && cols + P.lev_tau[levs[j]] > kmax) break;
            cols += P.lev_tau[levs[j]];
            ++k_last;
        }
    }
    while (i < nl) {
        const int rest = nl - i;
        const int k = rest <= k_last ? rest : 1;
        group[ng++] = k;
        i += k;
    }
    if (ng > kMaxPasses) return;
    long long xrow = 0, arow = 0;
    const long long n_root = 1LL << (P.m - P.JF);
    for (int g = 0, li = 0; g < ng; ++g) {
        LevelPass& ps = L.pass[g];
        ps = LevelPass{};
        ps.nseg = group[g];
        int lowest = 0;
        for (int k = 0; k < ps.nseg; ++k, ++li) {
            const int I = levs[li];
            LevelSeg& sg = ps.seg[k];
            sg.level = I;
            sg.chunks = (P.lev_tau[I] + 31) / 32;
            sg.last_ksteps = (P.lev_tau[I] - 32 * (sg.chunks - 1) + 15) / 16;
            sg.logn = P.m - I;
            sg.logn_rep = std::max(P.m - I, 7);
            sg.col0 = P.lev_col0[I];
            sg.tau = P.lev_tau[I];
            sg.tab = P.lev_tab[I];
            sg.xrow = xrow;
            sg.arow = arow;
            xrow += (long long)L.pieces * sg.chunks << sg.logn_rep;
            arow += (long long)L.pieces * sg.chunks * L.tA;
            lowest = std::max(lowest, sg.logn);
        }
        ps.logn_out = g + 1 == ng ? P.m - P.JF : lowest;
        ps.logn_next = g == 0 ? -1 : L.pass[g - 1].logn_out;
        const long long n_out = 1LL << ps.logn_out;
        ps.rho_tiles = (int)std::max(1LL, n_out / 128);
        ps.t_tiles = t_tiles;
        ps.reps = 1;
        if (ps.logn_next >= 7 && ps.logn_out > ps.logn_next) ps.reps = 1 << (ps.logn_out - ps.logn_next);
        ps.ntiles = (long long)ps.rho_tiles * ps.t_tiles * P.reff;
    }
    (void)n_root;
    // TMA coordinates are 32-bit
    if (xrow >= (1LL << 31) || arow >= (1LL << 31)) return;
    L.npass = ng;
    L.x_rows_per_shift = xrow;
    L.a_rows = arow;
    P.lv = true;
}

// The plan of a rule in a prime base b > 2: the generic top-down levels on the CUDA cores (every
// tier; the tensor-core tiers compute in FP32), no binary fine band (the last level is written at
// all N rows), the integrand row by row, and the adjoint's folds and block gradients per level.
qmc_status make_plan_b(int op, const qmc_rule* r, uint32_t tau, const qmc_integrand* f, int precision,
                       const void* d_A, Plan& P) {
    P.op = op;
    P.base_b = true;
    P.b = (int)r->b;
    P.kind = r->kind; P.m = (int)r->m; P.s = (int)r->s; P.transform = r->transform;
    P.R = (int)r->R; P.reff = std::max(P.R, 1);
    for (int I = 0; I <= P.m; ++I) {
        long long n = 1;
        for (int i = 0; i < P.m - I; ++i) n *= P.b;
        P.lev_n[I] = n;
        P.lev_tau[I] = 0;
        P.lev_col0[I] = -1;
    }
    P.N = P.lev_n[0];
    for (int j = 0; j < P.s; ++j) {
        const int I = (int)std::min<uint32_t>(r->w[j], r->m);
        if (P.lev_col0[I] < 0) P.lev_col0[I] = j;
        P.lev_tau[I]++;
    }
    {
        int next = P.s;
        for (int I = P.m; I >= 0; --I) {
            if (P.lev_col0[I] < 0) P.lev_col0[I] = next;
            else next = P.lev_col0[I];
        }
    }
    P.lev_tab[0] = 0;
    for (int I = 0; I <= P.m; ++I) P.lev_tab[I + 1] = P.lev_tab[I] + (long long)P.lev_tau[I] * P.lev_n[I];
    P.T_tot = P.lev_tab[P.m + 1];
    P.tab_stride = (P.T_tot + 3) / 4 * 4;
    P.need_gen = (r->d_gen == nullptr);
    P.has_shift = P.kind != QMC_REDUCED_MC && P.R > 0;
    P.need_shift = (P.has_shift && r->d_shift == nullptr);
    size_t off = 0;
    P.off_gen = off;
    if (P.need_gen) off = align256(off + sizeof(uint32_t) * gen_words(P));
    P.off_shift = off;
    if (P.need_shift) off = align256(off + sizeof(uint32_t) * (size_t)P.R * P.s);
    if (op == QMC_OP_GEN_POINTS) { P.total = off; return QMC_OK; }
    if (precision != QMC_FP64 && precision != QMC_FP32 && precision != QMC_SPLIT && precision != QMC_BF16)
        return fail(QMC_ERR_INVALID_ARG, "precision %d unknown", precision);
    if (tau < 1 || tau > 65536) return fail(QMC_ERR_INVALID_ARG, "tau=%u outside [1, 65536]", tau);
    P.precision = precision;
    P.tc_pieces = 0;
    P.elt = precision == QMC_FP64 ? 8 : 4;
    P.tau = (int)tau;
    P.tau_pad = (int)((tau + 3) / 4 * 4);
    if (op == QMC_OP_INTEGRATE || op == QMC_OP_INTEGRATE_BWD) {
        if (!f) return fail(QMC_ERR_INVALID_ARG, "integrand is NULL");
        if (f->kind < QMC_F_LINEAR_MEAN || f->kind > QMC_F_LOGSUMEXP)
            return fail(QMC_ERR_INVALID_ARG, "integrand kind %d unknown (QMC_F_NONE is only for the product)", f->kind);
        P.fkind = f->kind;
    }
    P.JF = 0;
    P.cg_count = 1;
    P.bl_n = 0;
    for (int I = P.m; I >= 0; --I)
        if (P.lev_tau[I] > 0) P.bl_lev[P.bl_n++] = I;
    for (int q = 0; q < P.bl_n; ++q) P.bl_rows[q] = q + 1 == P.bl_n ? P.N : P.lev_n[P.bl_lev[q]];
    {
        const long long rpt = std::max(1LL, std::min(16LL, P.N * P.reff / (152LL * 8 * 256 * 4)));
        P.nblk = (int)((P.N + 256 * rpt - 1) / (256 * rpt));
    }
    const size_t E = (size_t)P.elt;
    P.need_pad = !((tau % 4) == 0 && d_A != nullptr && (((uintptr_t)d_A) % 16) == 0);
    P.off_A = off;
    if (P.need_pad) off = align256(off + E * (size_t)P.s * P.tau_pad);
    P.off_tab = off;
    off = align256(off + E * (size_t)P.reff * P.tab_stride);
    const bool fused = op == QMC_OP_INTEGRATE || op == QMC_OP_INTEGRATE_BWD;
    P.S_per_shift = P.N * P.tau_pad;
    P.off_S = off;
    if (fused && P.bl_n) off = align256(off + E * (size_t)P.reff * P.S_per_shift);
    if (fused) {
        P.off_rowsave = off;
        off = align256(off + 2 * E * (size_t)P.reff * P.N);
        P.off_fpart = off;
        off = align256(off + sizeof(double) * (size_t)P.reff * P.nblk);
        P.off_ticket = off;
        off = align256(off + sizeof(unsigned int));
    }
    // shared region: the levels' partial sums (dead after the last level), the row partials, then
    // the backward's gradients
    const size_t u0 = off;
    size_t uend = u0, o = u0;
    for (int q = 0; q + 1 < P.bl_n; ++q) {
        P.bl_out[q] = o;
        o = align256(o + E * (size_t)P.reff * (size_t)P.bl_rows[q] * P.tau_pad);
    }
    if (P.bl_n) P.bl_out[P.bl_n - 1] = P.off_S;
    uend = std::max(uend, o);
    if (fused) {
        o = u0;
        P.off_rowpart = o;
        o = align256(o + E * (size_t)P.reff * P.N);
        P.off_rowmax = o;
        if (P.fkind == QMC_F_LOGSUMEXP) o = align256(o + E * (size_t)P.reff * P.N);
        uend = std::max(uend, o);
    }
    if (op == QMC_OP_INTEGRATE_BWD) {
        o = u0;
        P.off_G = o;
        o = align256(o + E * (size_t)P.reff * (size_t)P.N * P.tau_pad);
        // F of every level, from the lowest up (the lowest level's F is G itself when it has N rows)
        P.chb = Chain{};
        long long poff = 0;
        for (int q = P.bl_n - 1; q >= 0; --q) {
            const int I = P.bl_lev[q];
            const long long n = P.lev_n[I];
            if (n == P.N) P.bl_F[q] = P.off_G;
            else {
                P.bl_F[q] = o;
                o = align256(o + E * (size_t)P.reff * (size_t)n * P.tau_pad);
            }
            const long long K = (long long)P.reff * n;
            long long split = std::min(4096LL, (K + 8191) / 8192);
            P.bl_kper[q] = (K + split - 1) / split;
            P.bl_split[q] = (int)split;
            const int e = P.chb.count++;
            P.chb.col0[e] = P.lev_col0[I];
            P.chb.tau[e] = P.lev_tau[I];
            P.chb.split[e] = (int)split;
            P.chb.poff[e] = poff;
            poff += split * P.lev_tau[I] * P.tau_pad;
        }
        for (int q = 0; q < P.bl_n; ++q) P.bl_part[q] = 0;
        const size_t part0 = o;
        o = align256(o + E * (size_t)std::max(poff, 1LL));
        P.off_partc = part0;
        P.partc_elems = poff;
        P.groups = 1;
        P.kf_width = 1;
        P.off_gradpart = o;                  // (no fine band: one zero-sized partial)
        o = align256(o + E * (size_t)P.tau_pad);
        uend = std::max(uend, o);
    }
    P.total = uend;
    if (P.chb.count > kMaxChain) return fail(QMC_ERR_UNSUPPORTED, "too many weight levels");
    return QMC_OK;
}

qmc_status make_plan(int op, const qmc_rule* r, uint32_t tau, const qmc_integrand* f, int precision,
                     const void* d_A, Plan& P) {
    qmc_status st = validate(r);
    if (st != QMC_OK) return st;
    if (r->b > 2) return make_plan_b(op, r, tau, f, precision, d_A, P);
    P.op = op;
    P.kind = r->kind; P.m = (int)r->m; P.s = (int)r->s; P.transform = r->transform;
    P.R = (int)r->R; P.reff = std::max(P.R, 1);
    P.N = 1LL << P.m;
    P.nonper = net_nonperiodic(r);
    for (int I = 0; I <= P.m; ++I) { P.lev_tau[I] = 0; P.lev_col0[I] = -1; }
    for (int j = 0; j < P.s; ++j) {
        // (a non-periodic net has no distinct-row reuse: every column is on level 0)
        const int I = P.nonper ? 0 : (int)std::min<uint32_t>(r->w[j], r->m);
        if (P.lev_col0[I] < 0) P.lev_col0[I] = j;
        P.lev_tau[I]++;
    }
    {   // empty levels get the next column index (never read)
        int next = P.s;
        for (int I = P.m; I >= 0; --I) {
            if (P.lev_col0[I] < 0) P.lev_col0[I] = next;
            else next = P.lev_col0[I];
        }
    }
    P.xc = 0.0f;
    P.lev_tab[0] = 0;
    for (int I = 0; I <= P.m; ++I) P.lev_tab[I + 1] = P.lev_tab[I] + (long long)P.lev_tau[I] * (1LL << (P.m - I));
    P.T_tot = P.lev_tab[P.m + 1];
    P.tab_stride = (P.T_tot + 3) / 4 * 4;
    P.need_gen = (r->d_gen == nullptr);
    P.has_shift = P.kind != QMC_REDUCED_MC && P.R > 0;
    P.need_shift = (P.has_shift && r->d_shift == nullptr);

    size_t off = 0;
    P.off_gen = off;
    if (P.need_gen) off = align256(off + sizeof(uint32_t) * gen_words(P));
    P.off_shift = off;
    if (P.need_shift) off = align256(off + sizeof(uint32_t) * (size_t)P.R * P.s);
    if (op == QMC_OP_GEN_POINTS) { P.total = off; return QMC_OK; }

    if (precision != QMC_FP64 && precision != QMC_FP32 && precision != QMC_SPLIT && precision != QMC_BF16)
        return fail(QMC_ERR_INVALID_ARG, "precision %d unknown", precision);
    // the tensor-core tiers keep FP32 data and FP32 arithmetic outside the coarse block products
    P.tc_pieces = precision == QMC_SPLIT ? 3 : precision == QMC_BF16 ? 1 : 0;
    if (P.tc_pieces && (P.transform == QMC_T_IDENTITY || P.transform == QMC_T_TENT)) P.xc = 0.5f;
    if (tau < 1 || tau > 65536) return fail(QMC_ERR_INVALID_ARG, "tau=%u outside [1, 65536]", tau);
    P.precision = precision;
    P.elt = precision == QMC_FP64 ? 8 : 4;
    P.tau = (int)tau;
    P.tau_pad = (int)((tau + 3) / 4 * 4);
    if (op == QMC_OP_INTEGRATE || op == QMC_OP_INTEGRATE_BWD) {
        if (!f) return fail(QMC_ERR_INVALID_ARG, "integrand is NULL");
        if (f->kind < QMC_F_LINEAR_MEAN || f->kind > QMC_F_LOGSUMEXP)
            return fail(QMC_ERR_INVALID_ARG, "integrand kind %d unknown (QMC_F_NONE is only for the product)", f->kind);
        P.fkind = f->kind;
    }

    {   // the schedule cache's key: everything the fine schedules depend on
        std::string k = "m" + std::to_string(P.m) + " p" + std::to_string(precision) + " f" + std::to_string(P.fkind) +
                        " t" + std::to_string(P.tau_pad) + " r" + std::to_string(P.reff) + " L";
        for (int I = 0; I <= P.m; ++I) k += (I ? "," : "") + std::to_string(P.lev_tau[I]);
        P.tune_key = k;
        if (t_hint) {
            P.tuned = *t_hint;
        } else {
            TuneCache& tc = tune_cache();
            std::lock_guard<std::mutex> g(tc.mu);
            auto it = tc.m.find(k);
            if (it != tc.m.end()) P.tuned = it->second;
        }
    }
    // fine band shape
    auto fits = [&](int jf, const int* kmax) {
        if (P.m < jf) return false;
        for (int I = 0; I < jf; ++I)
            if (P.lev_tau[I] > kmax[I]) return false;
        return true;
    };
    const int k4[4] = {1, 2, 4, 8}, k1[1] = {16};
    if (precision != QMC_FP64 && fits(4, k4)) {
        P.shape = SHAPE_S4; P.JF = 4; P.kf_width = 15; P.cw_bwd = 2;
        P.exact = P.lev_tau[0] == 1 && P.lev_tau[1] == 2 && P.lev_tau[2] == 4 && P.lev_tau[3] == 8;
    }
    else if (fits(1, k1)) { P.shape = SHAPE_S1; P.JF = 1; P.kf_width = 16; P.cw_bwd = precision == QMC_FP64 ? 1 : 2; }
    else { P.shape = SHAPE_S0; P.JF = 0; P.kf_width = 0; P.cw_bwd = precision == QMC_FP64 ? 2 : 4; }
    const int logn_root = P.m - P.JF;
    const long long n_root = 1LL << logn_root;

    // coarse chain: levels JF..m with columns.  A level with many columns (a long K for its few
    // distinct rows) is cut into up to 8 column ranges, each its own entry with its own block
    // product, so that the levels run in parallel; the chain sum adds the entries' products.
    // (The tensor-core block products run long K well, so their levels are cut more coarsely.)
    const int cut_cols = P.tc_pieces ? 64 : 32;
    const int fwd_rows = P.tc_pieces ? tc_fwd_rows() : 64;
    int nsplit_tot = 0;
    for (int I = P.JF; I <= P.m; ++I)
        if (P.lev_tau[I] > 0) nsplit_tot += std::min(8, (P.lev_tau[I] + cut_cols - 1) / cut_cols);
    const bool cut = nsplit_tot <= kMaxChain;
    P.chf.count = 0;
    long long boff = 0;
    int tiles = 0;
    for (int I = P.JF; I <= P.m; ++I) {
        if (P.lev_tau[I] == 0) continue;
        const int parts = cut ? std::min(8, (P.lev_tau[I] + cut_cols - 1) / cut_cols) : 1;
        const int width = (P.lev_tau[I] + parts - 1) / parts;
        for (int pc = 0; pc < parts; ++pc) {
            const int c0 = pc * width, cw = std::min(width, P.lev_tau[I] - c0);
            if (cw <= 0) break;
            const int e = P.chf.count++;
            P.chf.lev[e] = I; P.chf.logn[e] = P.m - I; P.chf.tau[e] = cw; P.chf.col0[e] = P.lev_col0[I] + c0;
            P.chf.tab[e] = P.lev_tab[I] + ((long long)c0 << (P.m - I));
            P.chf.boff[e] = boff;
            boff += (1LL << (P.m - I)) * P.tau_pad;
            P.chf.tile0[e] = tiles;
            tiles += (int)(((1LL << (P.m - I)) + fwd_rows - 1) / fwd_rows);
            P.chf.split[e] = 1; P.chf.poff[e] = 0;
        }
    }
    P.chf.tile0[P.chf.count] = tiles;
    P.B_per_shift = boff;
    P.S_per_shift = P.chf.count ? n_root * P.tau_pad : 0;
    if (P.tc_pieces && P.chf.count) {
        // Level passes (Algorithm 2 top down) once the coarse partial sums are large enough for their
        // memory traffic to matter (each pass is one persistent launch with a fixed cost); below that
        // the block products and the chain sum.  A tuned schedule decides either way.
        long long partial = 0;
        for (int I = P.JF; I <= P.m; ++I)
            if (P.lev_tau[I] > 0) partial += (1LL << (P.m - I)) * P.tau_pad * P.reff;
        bool use = partial >= (1LL << 24);
        if (P.tuned.coarse == 1) use = true;
        if (P.tuned.coarse == 2) use = false;
        if (use) plan_levels(P);
    }

    // fine forward grid: 128 roots per CTA, column groups to fill the GPU
    P.root_blocks = (int)((n_root + 127) / 128);
    {
        const long long want = 4LL * 152;
        long long cg = (want + (long long)P.root_blocks * P.reff - 1) / ((long long)P.root_blocks * P.reff);
        cg = std::max(1LL, std::min(cg, (long long)(P.tau_pad + 15) / 16));
        cg = std::max(cg, (long long)(P.tau_pad + kMaxCR - 1) / kMaxCR);
        int cr = (int)((P.tau_pad + cg - 1) / cg);
        cr = std::min((cr + 15) / 16 * 16, kMaxCR);
        P.cr = cr;
        P.cg_count = (P.tau_pad + cr - 1) / cr;
    }
    // the S4 band of the float tiers: forward CTAs of 64 roots x 2 branches, column groups picked
    // by a per-SM cost model (CTAs per SM, at least the resident count, times columns per CTA plus a fixed
    // setup cost); the adjoint below.  m <= 27 keeps the adjoint's 32-bit staging offsets (4 * 2^m
    // table entries, 2 * 2^m row-save floats) below 2^30.
    P.fine_s4 = (op == QMC_OP_INTEGRATE || op == QMC_OP_INTEGRATE_BWD) && P.shape == SHAPE_S4 &&
                precision != QMC_FP64 && P.m <= 27;
    if (P.fine_s4) {
        // a thread per root (both level-3 nodes) for the integrands whose h needs few registers
        // (measured on the 2^20-point step: 4.56 -> 3.47 ms for the Gaussian norm, 3.29 -> 2.86 ms
        // for log-sum-exp); a thread per node otherwise; the schedule can pick either
        P.fwd_nb = (P.fkind == QMC_F_MEAN_COS || P.fkind == QMC_F_PDE_INV_SQ) ? 1 : 2;
        if (P.tuned.fwd_nb == 1 || P.tuned.fwd_nb == 2) P.fwd_nb = P.tuned.fwd_nb;
        const int rows = fine_s4_fwd_roots(P.fwd_nb);
        P.root_blocks = (int)((n_root + rows - 1) / rows);
        const long long rbr = (long long)P.root_blocks * P.reff;
        const int quads = P.tau_pad / 4, qmax = 512 / 4;
        const long long resident = fine_s4_fwd_resident(P.fkind, P.fwd_nb);
        long long best = -1;
        for (int cg = (quads + qmax - 1) / qmax; cg <= quads; ++cg) {
            const int qpg = (quads + cg - 1) / cg;
            if ((long long)(cg - 1) * qpg >= quads) continue;       // an empty last group
            const long long per_sm = (rbr * cg + 151) / 152;
            const long long cost = std::max(per_sm, resident) * (qpg + 2);
            if (best < 0 || cost < best) { best = cost; P.cr = 4 * qpg; P.cg_count = (quads + qpg - 1) / qpg; }
        }
        const int qpg = P.tuned.fwd_qpg;
        if (qpg > 0 && qpg <= qmax && qpg <= quads) { P.cr = 4 * qpg; P.cg_count = (quads + qpg - 1) / qpg; }
    }
    // the materialised product of the float tiers with the S4 band: CTAs of 256 columns over a
    // range of roots, as many as fill 5 CTAs per SM once (the band is bound by its output writes;
    // an even spread over the SMs matters more than whole batches of 8 roots); the band's 32-bit
    // staging offsets (below 4 * 2^m) need m <= 27
    P.fine_mat = op == QMC_OP_REDUCED_MATMUL && P.shape == SHAPE_S4 && precision != QMC_FP64 && P.m <= 27;
    if (P.fine_mat) {
        const int cols = fine_s4_mat_cols();
        P.passes = (P.tau_pad + cols - 1) / cols;
        const long long want = std::max(1LL, 152LL * 5 / ((long long)P.passes * P.reff));
        const long long rpc = std::max(1LL, (n_root + want - 1) / want);
        P.roots_per_cta = (int)rpc;
        P.groups = (int)((n_root + rpc - 1) / rpc);
    }
    // partials of the estimate: row blocks of the finalisation, 256 threads of rpt rows each (one
    // row per thread up to about four waves of 8 CTAs per SM, then up to 16 rows per thread)
    {
        const long long rpt = std::max(1LL, std::min(16LL, P.N * P.reff / (152LL * 8 * 256 * 4)));
        P.nblk = (int)((P.N + 256 * rpt - 1) / (256 * rpt));
    }

    // backward schedule
    if (op == QMC_OP_INTEGRATE_BWD && P.fine_s4) {
        // 256 columns per CTA; an even number of roots per CTA (the two halves take alternate
        // roots), chosen by the same kind of cost model (at least 2 CTAs of 8 warps resident per
        // SM, a fixed setup cost of about 8 roots per CTA)
        // two column pairs per lane: every broadcast load of a root's staged x values feeds twice the
        // FP32 work, at one CTA of 8 warps per SM (measured on the 2^20-point step: 8.43 -> 7.65 ms)
        P.bwd_cpl = P.tuned.bwd_cpl == 1 ? 1 : 2;
        const int cols = fine_s4_bwd_cols(P.bwd_cpl), rb = fine_s4_bwd_batch();
        const long long resident = P.bwd_cpl == 2 ? 1 : 2;     // CTAs of 8 warps per SM
        P.passes = (P.tau_pad + cols - 1) / cols;
        long long best = -1;
        const long long gmax = std::min<long long>((n_root + 1) / 2, 152LL * 16);
        for (long long G = 1; G <= gmax; ++G) {
            const long long rpc = ((n_root + G - 1) / G + 1) / 2 * 2;
            const long long g = (n_root + rpc - 1) / rpc;
            if (g != G) continue;
            const long long per_sm = ((long long)P.passes * g * P.reff + 151) / 152;
            const long long cost = std::max(per_sm, resident) * (rpc + rb);
            if (best < 0 || cost < best) { best = cost; P.roots_per_cta = (int)rpc; P.groups = (int)g; }
        }
        const long long rpc = P.tuned.bwd_rpc;
        if (rpc >= 2 && rpc % 2 == 0 && rpc <= n_root + 1) {
            P.roots_per_cta = (int)rpc;
            P.groups = (int)((n_root + rpc - 1) / rpc);
        }
    }
    if (op == QMC_OP_INTEGRATE_BWD) {
        if (!P.fine_s4) {
            const int cols_per_pass = 32 * P.cw_bwd;
            P.passes = (P.tau_pad + cols_per_pass - 1) / cols_per_pass;
            long long groups_target = std::max(1LL, 304LL / ((long long)P.passes * P.reff));
            long long rpc = (n_root + groups_target - 1) / groups_target;
            rpc = std::max(rpc, (n_root + 511) / 512);
            rpc = std::max(8LL, (rpc + 7) / 8 * 8);
            P.roots_per_cta = (int)rpc;
            P.groups = (int)((n_root + rpc - 1) / rpc);
        }
        // Root gradients are folded level by level (k_fold_tree) up to I_mat = the highest coarse
        // level below m within kFoldDepth of the root; F of every coarse level up to I_mat is
        // materialised, the levels above it (the constant level m) fold from F_{I_mat} on the fly.
        P.chb = P.chf;
        if (P.tc_pieces != 0) {
            // the tensor-core gradients take up to 128 columns of a level per entry (MMA N)
            Chain c{};
            for (int e = 0; e < P.chf.count; ++e) {
                const int I = P.chf.lev[e];
                if (e > 0 && P.chf.lev[e - 1] == I) continue;      // the level's first entry only
                const int parts = (P.lev_tau[I] + 127) / 128, width = (P.lev_tau[I] + parts - 1) / parts;
                for (int pc = 0; pc < parts; ++pc) {
                    const int c0 = pc * width, cw = std::min(width, P.lev_tau[I] - c0);
                    if (cw <= 0) break;
                    const int f = c.count++;
                    c.lev[f] = I; c.logn[f] = P.m - I; c.tau[f] = cw; c.col0[f] = P.lev_col0[I] + c0;
                    c.tab[f] = P.lev_tab[I] + ((long long)c0 << (P.m - I));
                    c.split[f] = 1;
                }
            }
            P.chb = c;
        }
        const int max_depth = precision == QMC_FP64 ? 5 : 6;
        int I_mat = P.JF;
        for (int e = 0; e < P.chb.count; ++e)
            if (P.chb.lev[e] < P.m && P.chb.lev[e] - P.JF <= max_depth) I_mat = std::max(I_mat, P.chb.lev[e]);
        P.fold.depth = I_mat - P.JF;
        P.fold.logn_top = P.m - I_mat;
        for (int d = 0; d < 8; ++d) { P.fold.want[d] = 0; P.fold.off[d] = 0; }
        long long fchain = 0;
        for (int e = 0; e < P.chb.count; ++e) {
            const int I = P.chb.lev[e];
            if (I > P.JF && I <= I_mat) {
                if (!P.fold.want[I - P.JF]) {        // one folded buffer per level, shared by its entries
                    P.fold.want[I - P.JF] = 1;
                    P.fold.off[I - P.JF] = fchain;
                    fchain += (1LL << (P.m - I)) * P.tau_pad;
                }
                P.chb.fsel[e] = 1; P.chb.foff[e] = P.fold.off[I - P.JF]; P.chb.flog[e] = 0;
            }
        }
        for (int e = 0; e < P.chb.count; ++e) {
            const int I = P.chb.lev[e];
            if (I == P.JF) { P.chb.fsel[e] = 0; P.chb.foff[e] = 0; P.chb.flog[e] = 0; }
            else if (I > I_mat) {
                P.chb.fsel[e] = I_mat > P.JF ? 1 : 0;
                P.chb.foff[e] = I_mat > P.JF ? P.fold.off[I_mat - P.JF] : 0;
                P.chb.flog[e] = I - I_mat;
            }
        }
        // a level above JF that has no columns but is the fold top still needs its rows
        if (I_mat > P.JF && !P.fold.want[I_mat - P.JF]) {
            P.fold.want[I_mat - P.JF] = 1;
            P.fold.off[I_mat - P.JF] = fchain;
            fchain += (1LL << (P.m - I_mat)) * P.tau_pad;
        }
        // the lowest coarse levels fused with the fold: L levels JF .. JF+L-1, each with at most one
        // entry of at most 64 columns (read from its materialised fold), F_{JF+L} materialised with
        // at least 32 rows, at most 128 accumulator columns in all
        P.fg_L = 0;
        for (int d = 0; d < kMaxFoldLv; ++d) P.fg_ent[d] = -1;
        // the fused kernel and k_grad_tc pay their fixed costs (tensor-memory set-up, two producer
        // warps, the pre-split pass) once the root gradients reach 2^24 elements; below that one
        // fold kernel and k_coarse_grad_tc take every level
        P.bwd_tma = P.tc_pieces != 0 && (P.tuned.bwd == 2 ||
                                         (P.tuned.bwd == 0 && (long long)P.reff * n_root * P.tau_pad >= (1LL << 24)));
        if (P.bwd_tma && !P.nonper && precision != QMC_FP64) {
            for (int L = kMaxFoldLv; L >= 1 && P.fg_L == 0; --L) {
                if (P.JF + L > I_mat || P.m - (P.JF + L) < 5) continue;
                int ent[kMaxFoldLv] = {-1, -1, -1}, ncols = 0, good = 1, any = 0;
                for (int e = 0; e < P.chb.count; ++e) {
                    const int d = P.chb.lev[e] - P.JF;
                    if (d < 0 || d >= L) continue;
                    if (ent[d] >= 0 || P.chb.flog[e] != 0 || P.chb.tab[e] % 4 != 0) good = 0;
                    ent[d] = e;
                    ncols += (P.chb.tau[e] + 15) / 16 * 16;
                    any = 1;
                }
                if (!good || !any || ncols > 128 || P.tab_stride % 4 != 0) continue;
                P.fg_L = L;
                for (int d = 0; d < L; ++d) P.fg_ent[d] = ent[d];
            }
        }
        P.froot_tiled = P.fg_L > 0 && P.fine_s4;
        if (P.fg_L) {
            const int L = P.fg_L;
            if (!P.fold.want[L]) {          // F_{JF+L} is the fused kernel's output
                P.fold.want[L] = 1;
                P.fold.off[L] = fchain;
                fchain += (1LL << (P.m - P.JF - L)) * P.tau_pad;
            }
            P.fold2 = FoldLevels{};
            P.fold2.depth = P.fold.depth - L;
            P.fold2.logn_top = P.fold.logn_top;
            for (int d = 1; d <= P.fold2.depth; ++d) {
                P.fold2.want[d] = P.fold.want[L + d];
                P.fold2.off[d] = P.fold.off[L + d];
            }
        }
        P.Fchain_per_shift = fchain;
        // coarse gradient GEMMs: K = R n_e rows; splits balance the work over the GPU.  FP32/FP64
        // tiles: 16 columns j, 16 multiply-adds plus 4 fold loads per K row and column, ~4 CTAs
        // per SM.  Tensor-core tiles: 64 columns j, work ~ the operand loads (2 + fold per K row
        // and column), ~3 CTAs per SM and at least 128 K rows per split.
        const bool tc = P.tc_pieces != 0;
        const int jcols = tc ? tc_grad_cols() : 16;
        // (the tensor-core kernel runs one CTA per SM: about one wave of 152 CTAs)
        const double fma_w = tc ? 2.0 : 16.0, fold_w = tc ? 1.0 : 4.0, target = tc ? 152.0 : 608.0;
        const long long kmin = tc ? 128 : 64;
        const int ttiles = (P.tau_pad + 127) / 128;
        auto fused = [&](int e) {
            for (int d = 0; d < P.fg_L; ++d)
                if (P.fg_ent[d] == e) return true;
            return false;
        };
        // the fused kernel: one CTA per SM, each on a column tile and a range of (shift, residue
        // block) items; its partials are split over the CTAs of a column tile
        const int fg_cpt = P.fg_L ? (int)std::max(1LL, std::min<long long>(152 / ttiles,
                                         (long long)P.reff << (P.m - P.JF - P.fg_L - 5))) : 0;
        double wtot = 0.0;
        for (int e = 0; e < P.chb.count; ++e) {
            if (fused(e)) continue;
            const long long K = (long long)P.reff << (P.m - P.chb.lev[e]);
            const double fold = (double)(1LL << P.chb.flog[e]);
            wtot += (double)((P.chb.tau[e] + jcols - 1) / jcols) * ttiles * K * (fma_w + fold_w * fold);
        }
        long long poff = 0;
        int bt = 0;
        for (int e = 0; e < P.chb.count; ++e) {
            if (fused(e)) {
                P.chb.kper[e] = 0;
                P.chb.split[e] = fg_cpt;
                P.chb.poff[e] = poff;
                poff += (long long)fg_cpt * P.chb.tau[e] * P.tau_pad;
                P.chb.tile0[e] = bt;
                continue;
            }
            const long long K = (long long)P.reff << (P.m - P.chb.lev[e]);
            const double fold = (double)(1LL << P.chb.flog[e]);
            const int jt = (P.chb.tau[e] + jcols - 1) / jcols;
            const double we = (double)jt * ttiles * K * (fma_w + fold_w * fold);
            long long split = (long long)(we / std::max(wtot, 1.0) * target / ((double)jt * ttiles) + 0.5);
            split = std::max(1LL, std::min(split, std::max(1LL, K / kmin)));
            // tensor-core splits of at most 4096 rows: an FP32 accumulator in tensor memory then sums
            // at most 1024 rows (four per CTA), and the splits are summed in double
            if (tc) split = std::max(split, (K + 1023) / 1024);
            split = std::min(split, 4096LL);
            long long kper = (K + split - 1) / split;
            if (tc) {                       // whole chunks of 32 rows per split
                kper = (kper + 31) / 32 * 32;
                split = (K + kper - 1) / kper;
            }
            P.chb.kper[e] = kper;
            P.chb.split[e] = (int)split;
            P.chb.poff[e] = poff;
            poff += split * P.chb.tau[e] * P.tau_pad;
            P.chb.tile0[e] = bt;
            bt += jt * (int)split;
        }
        P.chb.tile0[P.chb.count] = bt;
        P.bwd_tiles = bt;
        P.partc_elems = poff;
        P.ngsel = 0;
        P.chl = P.chb;
        P.chl.count = 0;
        int btl = 0;
        for (int e = 0; e < P.chb.count; ++e) {
            if (fused(e)) continue;
            const bool tma = P.bwd_tma && P.chb.flog[e] == 0 && P.m - P.chb.lev[e] >= 5 && P.chb.tab[e] % 4 == 0 &&
                             P.chb.tau[e] <= 128 &&
                             P.chb.foff[e] % 4 == 0 && P.tau_pad % 4 == 0 && P.tab_stride % 4 == 0 &&
                             P.chb.kper[e] % 32 == 0 && P.ngsel < kMaxGradTc;
            if (tma) { P.gsel[P.ngsel++] = e; continue; }
            const int l = P.chl.count++;
            P.chl.lev[l] = P.chb.lev[e];
            P.chl.logn[l] = P.chb.logn[e]; P.chl.tau[l] = P.chb.tau[e]; P.chl.col0[l] = P.chb.col0[e];
            P.chl.tab[l] = P.chb.tab[e]; P.chl.boff[l] = P.chb.boff[e];
            P.chl.split[l] = P.chb.split[e]; P.chl.kper[l] = P.chb.kper[e]; P.chl.poff[l] = P.chb.poff[e];
            P.chl.fsel[l] = P.chb.fsel[e]; P.chl.flog[l] = P.chb.flog[e]; P.chl.foff[l] = P.chb.foff[e];
            P.chl.tile0[l] = btl;
            btl += (P.chb.tau[e] + jcols - 1) / jcols * P.chb.split[e];
        }
        P.chl.tile0[P.chl.count] = btl;
        P.bwd_tiles_l = btl;
        SplitXtArgs& sx = P.sxa;
        sx = SplitXtArgs{};
        long long xoff = 0;
        auto add_xt = [&](int e, int d) {
            const int l = sx.n++;
            sx.lev[l] = d;
            sx.logn[l] = P.chb.logn[e];
            sx.tau[l] = P.chb.tau[e];
            sx.tab[l] = P.chb.tab[e];
            sx.off[l] = xoff;
            sx.blk0[l + 1] = sx.blk0[l] + ((long long)P.chb.tau[e] << (P.chb.logn[e] - 3));
            xoff += (long long)P.tc_pieces * P.reff * P.chb.tau[e] << P.chb.logn[e];
            return sx.off[l];
        };
        if (P.fg_L) {
            const int L = P.fg_L;
            FoldGradArgs& g = P.fga;
            g = FoldGradArgs{};
            g.log_out = P.m - P.JF - L;
            g.items = (long long)P.reff << (g.log_out - 5);
            g.tau_pad = P.tau_pad;
            g.t_tiles = ttiles;
            g.cpt = fg_cpt;
            g.group = std::max(1, 32 >> L);            // level JF's chains: 32 2^L rows per item, <= 1024
            g.fout_stride = P.Fchain_per_shift;
            g.froot_tiled = P.froot_tiled ? 1 : 0;
            int acc = 0;
            for (int d = 0; d < L; ++d) {
                const int e = P.fg_ent[d];
                g.nd[d] = e >= 0 ? (P.chb.tau[e] + 15) / 16 * 16 : 0;
                g.tau[d] = e >= 0 ? P.chb.tau[e] : 0;
                g.acc[d] = acc;
                g.poff[d] = e >= 0 ? P.chb.poff[e] : 0;
                acc += g.nd[d];
                if (e >= 0) add_xt(e, d);
            }
            g.nt = 32;
            while (g.nt < acc) g.nt *= 2;
        }
        for (int i = 0; i < P.ngsel; ++i) P.gxoff[i] = add_xt(P.gsel[i], -1);
        P.xt_bytes = (size_t)xoff * 2;
    }

    // workspace layout
    const size_t E = (size_t)P.elt;
    P.need_pad = !((tau % 4) == 0 && d_A != nullptr && (((uintptr_t)d_A) % 16) == 0);
    P.off_A = off;
    if (P.need_pad) off = align256(off + E * (size_t)P.s * P.tau_pad);
    // areas that live through a whole forward (and, reused, the backward): the point table,
    // the root values and the per-row results
    P.off_tab = off;
    off = align256(off + E * (size_t)P.reff * P.tab_stride);
    P.off_S = off;
    off = align256(off + E * (size_t)P.reff * P.S_per_shift);
    if (op == QMC_OP_INTEGRATE || op == QMC_OP_INTEGRATE_BWD) {
        P.off_rowsave = off;
        off = align256(off + 2 * E * (size_t)P.reff * P.N);
        P.off_fpart = off;
        off = align256(off + sizeof(double) * (size_t)P.reff * P.nblk);
        P.off_ticket = off;
        off = align256(off + sizeof(unsigned int));
    }
    // one region shared by areas whose lives do not overlap on the stream: the coarse block
    // products (dead once summed into S), the row partials of the fused forward, and the
    // backward's gradient buffers
    const size_t u0 = off;
    size_t uend = u0;
    P.off_B = u0;
    if (P.lv) {
        // X pieces, A pieces, then the outputs of every pass but the last (which writes S)
        LevelPlan& L = P.lvp;
        size_t o = u0;
        L.x_off = o;
        o = align256(o + (size_t)P.reff * (size_t)L.x_rows_per_shift * 64);
        L.a_off = o;
        o = align256(o + (size_t)L.a_rows * 64);
        L.c_off = o;
        o = align256(o + 4 * (size_t)P.tau_pad);
        L.cpart_off = o;
        if (P.xc != 0.0f) o = align256(o + sizeof(double) * 64 * (size_t)P.tau_pad);
        L.xc = P.xc;
        for (int q = 0; q < L.npass; ++q) L.pass[q].const_off = -1;
        if (P.xc != 0.0f) L.pass[0].const_off = (long long)(L.c_off / 4);
        for (int q = 0; q + 1 < L.npass; ++q) {
            LevelPass& ps = L.pass[q];
            ps.out_off = (long long)(o / 4);
            ps.out_stride = (1LL << ps.logn_out) * P.tau_pad;
            o = align256(o + 4 * (size_t)P.reff * (size_t)ps.out_stride);
        }
        LevelPass& last = L.pass[L.npass - 1];
        last.out_off = (long long)(P.off_S / 4);
        last.out_stride = P.S_per_shift;
        for (int q = 1; q < L.npass; ++q) {
            L.pass[q].next_off = L.pass[q - 1].out_off;
            L.pass[q].next_stride = L.pass[q - 1].out_stride;
        }
        uend = std::max(uend, o);
    } else {
        uend = std::max(uend, align256(u0 + E * (size_t)P.reff * P.B_per_shift));
    }
    if (op == QMC_OP_INTEGRATE || op == QMC_OP_INTEGRATE_BWD) {
        size_t o = u0;
        P.off_rowpart = o;
        o = align256(o + E * (size_t)P.reff * P.cg_count * P.N);
        P.off_rowmax = o;
        if (P.fkind == QMC_F_LOGSUMEXP) o = align256(o + E * (size_t)P.reff * P.cg_count * P.N);
        uend = std::max(uend, o);
    }
    if (op == QMC_OP_INTEGRATE_BWD) {
        size_t o = u0;
        P.off_F = o;
        o = align256(o + E * (size_t)P.reff * (size_t)n_root * root_cols(P));
        P.off_Fchain = o;
        o = align256(o + E * (size_t)P.reff * (size_t)std::max(P.Fchain_per_shift, 1LL));
        P.off_gradpart = o;
        o = align256(o + E * (size_t)P.reff * P.groups * std::max(P.kf_width, 1) * P.tau_pad);
        P.off_partc = o;
        o = align256(o + E * (size_t)std::max(P.partc_elems, 1LL));
        P.off_gsum = o;
        if (P.xc != 0.0f) o = align256(o + sizeof(double) * 65 * (size_t)P.tau_pad);
        P.off_xt = o;
        o = align256(o + P.xt_bytes);
        uend = std::max(uend, o);
    }
    P.total = uend;
    return QMC_OK;
}

DevRule dev_rule(const Plan& P, const qmc_rule* r, char* ws) {
    DevRule R{};
    R.kind = P.kind; R.m = P.m; R.s = P.s; R.transform = P.transform; R.R = P.R;
    R.gen = P.need_gen ? reinterpret_cast<const uint32_t*>(ws + P.off_gen) : r->d_gen;
    R.shift = !P.has_shift ? nullptr : (P.need_shift ? reinterpret_cast<const uint32_t*>(ws + P.off_shift) : r->d_shift);
    R.T_tot = P.T_tot;
    R.nlev = P.m + 1;
    for (int I = 0; I <= P.m; ++I) { R.lev_tau[I] = P.lev_tau[I]; R.lev_col0[I] = P.lev_col0[I]; }
    for (int I = 0; I <= P.m + 1; ++I) R.lev_tab[I] = P.lev_tab[I];
    R.b = P.b;
    for (int I = 0; I <= P.m; ++I) R.lev_n[I] = P.base_b ? P.lev_n[I] : (1LL << (P.m - I));
    R.nonper = P.nonper ? 1 : 0;
    R.nw = 0;
    if (P.nonper) {
        for (int j = 0; j < P.s; ++j) {
            const int v = (int)std::min<uint32_t>(r->w[j], r->m);
            if (R.nw == 0 || R.wval[R.nw - 1] != v) { R.wcol0[R.nw] = j; R.wval[R.nw] = v; ++R.nw; }
        }
        R.wcol0[R.nw] = P.s;
    }
    return R;
}

qmc_status upload_rule(const Plan& P, const qmc_rule* r, char* ws, cudaStream_t st) {
    if (P.need_gen) {
        QMC_CUDA(cudaMemcpyAsync(ws + P.off_gen, P.kind == QMC_DIGITAL_NET ? r->C : r->z, gen_words(P) * 4,
                                 cudaMemcpyHostToDevice, st));
    }
    if (P.need_shift)
        QMC_CUDA(cudaMemcpyAsync(ws + P.off_shift, r->shift, (size_t)P.R * P.s * 4, cudaMemcpyHostToDevice, st));
    return QMC_OK;
}

// the integrand's pre-scale kappa (v = kappa y) and derivative factor (see Fn in qmc_internal.cuh)
double kappa_of(int F, double c) {
    return F == QMC_F_CALL_MEAN_EXP ? c * kLog2e : F == QMC_F_LOGSUMEXP ? kLog2e : 1.0;
}
double gfac_of(int F, double c) { return F == QMC_F_CALL_MEAN_EXP ? c : 1.0; }

template <class T>
FineArgs<T> fine_args(const Plan& P, char* ws, const T* A, int ldA, const qmc_integrand* f) {
    FineArgs<T> a{};
    a.tab = reinterpret_cast<const T*>(ws + P.off_tab);
    a.tab_stride = P.tab_stride;
    a.A = A; a.ldA = ldA;
    a.tau = P.tau; a.tau_pad = P.tau_pad;
    a.logn_root = P.m - P.JF;
    for (int I = 0; I < 4; ++I) {
        const bool in = I < P.JF;
        a.lev_tau[I] = in ? P.lev_tau[I] : 0;
        a.lev_col0[I] = in ? P.lev_col0[I] : 0;
        a.lev_logn[I] = in ? P.m - I : 0;
        a.lev_tab[I] = in ? P.lev_tab[I] : 0;
    }
    a.S = P.chf.count ? reinterpret_cast<const T*>(ws + P.off_S) : nullptr;
    a.S_stride = P.S_per_shift;
    a.cr = P.cr; a.cg_count = P.cg_count; a.reff = P.reff; a.r0 = 0;
    a.N = P.N;
    a.rowpart = reinterpret_cast<T*>(ws + P.off_rowpart);
    a.rowmax = reinterpret_cast<T*>(ws + P.off_rowmax);
    a.P = nullptr;
    a.c0 = f ? (T)f->params[0] : T(0);
    a.c1 = f ? (T)f->params[1] : T(0);
    a.tau_d = (double)P.tau;
    a.K_d = f ? f->params[1] : 0.0;
    a.fkind = P.fkind;
    a.kappa = (T)kappa_of(P.fkind, f ? f->params[0] : 0.0);
    return a;
}

// base b > 2: the table, the levels top down (the last at all N rows: the root values, or the
// product itself when materialised), then the integrand's row sums and the finalisation
template <class T>
qmc_status run_forward_b(const Plan& P, const qmc_rule* r, const T* dA, char* ws, const qmc_integrand* f, int mode,
                         T* dP, T* rowf, double* est, cudaStream_t st, const T** Aused, int* ldA_used) {
    qmc_status s0 = upload_rule(P, r, ws, st);
    if (s0 != QMC_OK) return s0;
    const DevRule R = dev_rule(P, r, ws);
    const T* A = dA;
    int ldA = P.tau;
    if (P.need_pad) {
        T* Ap = reinterpret_cast<T*>(ws + P.off_A);
        QMC_LAUNCH(st, "k_pad_A", launch_pad_A<T>(dA, Ap, P.s, P.tau, P.tau_pad, st));
        A = Ap;
        ldA = P.tau_pad;
    }
    *Aused = A;
    *ldA_used = ldA;
    T* tab = reinterpret_cast<T*>(ws + P.off_tab);
    unsigned int* ticket = mode == MODE_FUSED ? reinterpret_cast<unsigned int*>(ws + P.off_ticket) : nullptr;
    QMC_LAUNCH(st, "k_table_b", launch_table_b<T>(R, tab, P.T_tot, P.tab_stride, P.reff, ticket, st));
    const bool mat = mode == MODE_MATERIALIZE;
    for (int q = 0; q < P.bl_n; ++q) {
        const int I = P.bl_lev[q];
        LevelB lv{I, P.lev_tau[I], P.lev_col0[I], P.lev_n[I], P.lev_tab[I], P.bl_rows[q], q ? P.bl_rows[q - 1] : 1};
        const bool last = q + 1 == P.bl_n;
        T* out = last && mat ? dP : reinterpret_cast<T*>(ws + P.bl_out[q]);
        const long long out_stride = last && mat ? P.N * P.tau : P.bl_rows[q] * P.tau_pad;
        const T* next = q ? reinterpret_cast<const T*>(ws + P.bl_out[q - 1]) : nullptr;
        QMC_LAUNCH(st, "k_level_b", launch_level_b<T>(tab, P.tab_stride, A, ldA, P.tau_pad, lv, out, out_stride, next,
                                                     q ? P.bl_rows[q - 1] * P.tau_pad : 0, last && mat, P.tau,
                                                     P.reff, st));
    }
    if (mat && P.bl_n == 0)                  // no columns with points: P = 0
        QMC_CUDA(cudaMemsetAsync(dP, 0, sizeof(T) * (size_t)P.reff * P.N * P.tau, st));
    if (mode == MODE_FUSED) {
        if (P.bl_n == 0) QMC_CUDA(cudaMemsetAsync(ws + P.off_S, 0, sizeof(T) * (size_t)P.reff * P.S_per_shift, st));
        T* rowpart = reinterpret_cast<T*>(ws + P.off_rowpart);
        T* rowmax = reinterpret_cast<T*>(ws + P.off_rowmax);
        const double c0 = f->params[0];
        QMC_LAUNCH(st, "k_rows_b", launch_rows_b<T>(reinterpret_cast<const T*>(ws + P.off_S), P.S_per_shift, P.N, P.tau,
                                                   P.fkind, kappa_of(P.fkind, c0), c0, rowpart, rowmax, P.reff, st));
        T* rowsave = reinterpret_cast<T*>(ws + P.off_rowsave);
        double* fpart = reinterpret_cast<double*>(ws + P.off_fpart);
        const double coef_scale = gfac_of(P.fkind, c0) / ((double)P.reff * (double)P.N);
        QMC_LAUNCH(st, "k_rows_finalize",
                   launch_rows_finalize<T>(rowpart, rowmax, 1, P.N, P.reff, P.fkind, (double)P.tau, c0, f->params[1],
                                           coef_scale, rowsave, rowf, fpart, P.nblk, ticket, est, st));
    }
    return QMC_OK;
}

// base b > 2 adjoint: G = f'(Y)/(R N) row by row, folded level by level from the lowest up, each
// level's block gradient X~_I^T F_I in row splits, and the fixed-order sum of the splits
template <class T>
qmc_status run_backward_b(const Plan& P, const qmc_rule* r, const T* dA, char* ws, const qmc_integrand* f,
                          const double* upstream, T* grad, bool reuse, cudaStream_t st) {
    const T* A;
    int ldA;
    if (!reuse) {
        qmc_status s0 = run_forward_b<T>(P, r, dA, ws, f, MODE_FUSED, nullptr, nullptr, nullptr, st, &A, &ldA);
        if (s0 != QMC_OK) return s0;
    }
    const double c0 = f->params[0];
    T* G = reinterpret_cast<T*>(ws + P.off_G);
    QMC_LAUNCH(st, "k_grad_rows_b",
               launch_grad_rows_b<T>(reinterpret_cast<const T*>(ws + P.off_S), P.S_per_shift, P.N, P.tau, P.tau_pad,
                                     P.fkind, kappa_of(P.fkind, c0), c0, reinterpret_cast<const T*>(ws + P.off_rowsave),
                                     upstream, G, P.reff, st));
    const T* tab = reinterpret_cast<const T*>(ws + P.off_tab);
    T* partc = reinterpret_cast<T*>(ws + P.off_partc);
    const T* prev = G;
    long long n_prev = P.N;
    for (int q = P.bl_n - 1, e = 0; q >= 0; --q, ++e) {
        const int I = P.bl_lev[q];
        const long long n = P.lev_n[I];
        T* F = reinterpret_cast<T*>(ws + P.bl_F[q]);
        if (n < n_prev) QMC_LAUNCH(st, "k_fold_b", launch_fold_b<T>(prev, n_prev, F, n, P.tau_pad, P.reff, st));
        LevelB lv{I, P.lev_tau[I], P.lev_col0[I], n, P.lev_tab[I], n, 1};
        QMC_LAUNCH(st, "k_grad_b", launch_grad_b<T>(tab, P.tab_stride, F, lv, P.bl_kper[q], P.bl_split[q], P.reff,
                                                   P.tau_pad, partc + P.chb.poff[e], st));
        prev = F;
        n_prev = n;
    }
    int koff[4] = {0, 0, 0, 0}, col0[4] = {0, 0, 0, 0}, taul[4] = {0, 0, 0, 0};
    QMC_LAUNCH(st, "k_grad_reduce",
               launch_grad_reduce<T>(reinterpret_cast<const T*>(ws + P.off_gradpart), 0, 1, koff, col0, taul, 0, partc,
                                     P.chb, P.tau, P.tau_pad, P.s, grad, nullptr, 0.0, st));
    return QMC_OK;
}

// forward through the fine kernel (fused or materialised); returns the A pointer/ld used
template <class T>
qmc_status run_forward(const Plan& P, const qmc_rule* r, const T* dA, char* ws, const qmc_integrand* f, int mode,
                       T* dP, T* rowf, double* est, cudaStream_t st, const T** Aused, int* ldA_used) {
    if (P.base_b) return run_forward_b<T>(P, r, dA, ws, f, mode, dP, rowf, est, st, Aused, ldA_used);
    qmc_status s0 = upload_rule(P, r, ws, st);
    if (s0 != QMC_OK) return s0;
    const DevRule R = dev_rule(P, r, ws);
    const T* A = dA;
    int ldA = P.tau;
    if (P.need_pad) {
        T* Ap = reinterpret_cast<T*>(ws + P.off_A);
        QMC_LAUNCH(st, "k_pad_A", launch_pad_A<T>(dA, Ap, P.s, P.tau, P.tau_pad, st));
        A = Ap;
        ldA = P.tau_pad;
    }
    *Aused = A;
    *ldA_used = ldA;
    T* tab = reinterpret_cast<T*>(ws + P.off_tab);
    unsigned int* ticket = mode == MODE_FUSED ? reinterpret_cast<unsigned int*>(ws + P.off_ticket) : nullptr;
    QMC_LAUNCH(st, "k_table", launch_table<T>(R, tab, P.T_tot, P.tab_stride, P.reff, ticket, st));
    if (P.chf.count && P.lv) {
        if constexpr (std::is_same<T, float>::value) {
            unsigned char* wsb = reinterpret_cast<unsigned char*>(ws);
            if (P.xc != 0.0f)
                QMC_LAUNCH(st, "k_const_row", launch_const_row(A, ldA, P.tau, P.tau_pad, P.lvp, wsb, st));
            QMC_LAUNCH(st, "k_split_a", launch_split_a(A, ldA, P.tau, P.lvp, wsb, st));
            QMC_LAUNCH(st, "k_split_x", launch_split_x(tab, P.tab_stride, P.lvp, P.reff, wsb, st));
            for (int q = 0; q < P.lvp.npass; ++q)
                QMC_LAUNCH(st, "k_level_tc", launch_level_pass(P.lvp, q, P.reff, P.tau_pad, wsb, st));
        }
    } else if (P.chf.count) {
        T* B = reinterpret_cast<T*>(ws + P.off_B);
        if (P.tc_pieces) {
            if constexpr (std::is_same<T, float>::value)
                QMC_LAUNCH(st, "k_coarse_fwd_tc", launch_coarse_fwd_tc(tab, P.tab_stride, A, ldA, P.tau_pad, P.chf, B,
                                                                       P.B_per_shift, P.reff, P.tc_pieces, st));
        } else {
            QMC_LAUNCH(st, "k_coarse_fwd", launch_coarse_fwd<T>(tab, P.tab_stride, A, ldA, P.tau_pad, P.chf, B,
                                                                P.B_per_shift, P.reff, st));
        }
        QMC_LAUNCH(st, "k_chain_sum", launch_chain_sum<T>(B, P.B_per_shift, P.chf, reinterpret_cast<T*>(ws + P.off_S),
                                                          P.S_per_shift, P.m - P.JF, P.tau_pad, P.reff, st));
    }
    FineArgs<T> a = fine_args<T>(P, ws, A, ldA, mode == MODE_FUSED ? f : nullptr);
    a.P = dP;
    if (mode == MODE_FUSED && P.fine_s4) {
        if constexpr (std::is_same<T, float>::value) {
            QMC_LAUNCH(st, "k_fine_fwd_s4", launch_fine_fwd_s4(a, P.fkind, P.fwd_nb, dim3(P.root_blocks, P.cg_count, P.reff), st));
        }
    } else if (mode == MODE_MATERIALIZE && P.fine_mat) {
        if constexpr (std::is_same<T, float>::value) {
            a.roots_per_cta = P.roots_per_cta;
            QMC_LAUNCH(st, "k_fine_mat_s4", launch_fine_mat_s4(a, dim3(P.groups, P.passes, P.reff), st));
        }
    } else {
        dim3 grid(P.root_blocks, P.cg_count, P.reff);
        QMC_LAUNCH(st, mode == MODE_FUSED ? "k_fine_fwd" : "k_fine_fwd_materialize",
                   launch_fine_fwd<T>(a, P.shape, P.exact, mode == MODE_FUSED ? P.fkind : 0, mode, grid, st));
    }
    if (mode == MODE_FUSED) {
        T* rowsave = reinterpret_cast<T*>(ws + P.off_rowsave);
        double* fpart = reinterpret_cast<double*>(ws + P.off_fpart);
        const double coef_scale = gfac_of(P.fkind, f->params[0]) / ((double)P.reff * (double)P.N);
        QMC_LAUNCH(st, "k_rows_finalize",
                   launch_rows_finalize<T>(a.rowpart, a.rowmax, P.cg_count, P.N, P.reff,
                                           P.fkind, (double)P.tau,
                                           f->params[0], f->params[1], coef_scale, rowsave, rowf, fpart, P.nblk,
                                           ticket, est, st));
    }
    return QMC_OK;
}

template <class T>
qmc_status run_backward(const Plan& P, const qmc_rule* r, const T* dA, char* ws, const qmc_integrand* f,
                        const double* upstream, T* grad, bool reuse, cudaStream_t st) {
    if (P.base_b) return run_backward_b<T>(P, r, dA, ws, f, upstream, grad, reuse, st);
    const T* A;
    int ldA;
    if (!reuse) {
        qmc_status s0 = run_forward<T>(P, r, dA, ws, f, MODE_FUSED, nullptr, nullptr, nullptr, st, &A, &ldA);
        if (s0 != QMC_OK) return s0;
    } else {
        A = P.need_pad ? reinterpret_cast<const T*>(ws + P.off_A) : dA;
        ldA = P.need_pad ? P.tau_pad : P.tau;
    }
    const long long n_root = 1LL << (P.m - P.JF);
    const long long root_stride = n_root * root_cols(P);
    T* Froot = reinterpret_cast<T*>(ws + P.off_F);
    FineArgs<T> a = fine_args<T>(P, ws, A, ldA, f);
    a.rowsave = reinterpret_cast<const T*>(ws + P.off_rowsave);
    a.upstream = upstream;
    a.Froot = Froot;
    a.froot_tiled = P.froot_tiled ? 1 : 0;
    a.froot_stride = root_stride;
    a.gradpart = reinterpret_cast<T*>(ws + P.off_gradpart);
    a.roots_per_cta = P.roots_per_cta;
    a.groups = P.groups;
    a.kf_actual = P.kf_width;
    const int nfine_part = P.reff * P.groups;
    if (P.fine_s4) {
        if constexpr (std::is_same<T, float>::value)
            QMC_LAUNCH(st, "k_fine_bwd_s4", launch_fine_bwd_s4(a, P.fkind, P.bwd_cpl, dim3(P.groups, P.passes, P.reff), st));
    } else {
        dim3 grid(P.groups, P.passes, P.reff);
        QMC_LAUNCH(st, "k_fine_bwd", launch_fine_bwd<T>(a, P.shape, P.exact, P.fkind, grid, st));
    }
    // coarse block gradients; each level folds the root gradients onto its distinct rows on the fly
    const T* tab = reinterpret_cast<const T*>(ws + P.off_tab);
    T* partc = reinterpret_cast<T*>(ws + P.off_partc);
    if (P.chb.count)
    {
        T* Fchain = reinterpret_cast<T*>(ws + P.off_Fchain);
        __nv_bfloat16* xt = reinterpret_cast<__nv_bfloat16*>(ws + P.off_xt);
        if constexpr (std::is_same<T, float>::value) {
            if (P.sxa.n)
                QMC_LAUNCH(st, "k_split_xt", launch_split_xt(tab, P.tab_stride, P.sxa, P.reff, P.tc_pieces, xt, P.xc, st));
        }
        if (P.fg_L) {
            if constexpr (std::is_same<T, float>::value) {
                // levels JF .. JF+L-1 and their folds in one pass; the rest fold from F_{JF+L}
                FoldGradArgs ga = P.fga;
                ga.fout = Fchain + P.fold.off[P.fg_L];
                ga.part = partc;
                QMC_LAUNCH(st, "k_fold_grad_tc",
                           launch_fold_grad_tc(ga, P.fg_L, Froot, root_stride, n_root, xt, P.sxa, P.reff,
                                               P.tc_pieces, st));
                if (P.fold2.depth > 0)
                    QMC_LAUNCH(st, "k_fold_tree",
                               launch_fold_tree<T>(Fchain + P.fold.off[P.fg_L], P.Fchain_per_shift, Fchain,
                                                   P.Fchain_per_shift, P.fold2, P.tau_pad, P.reff, st));
            }
        } else if (P.fold.depth > 0)
            QMC_LAUNCH(st, "k_fold_tree", launch_fold_tree<T>(Froot, root_stride, Fchain, P.Fchain_per_shift, P.fold,
                                                              P.tau_pad, P.reff, st));
        if (P.tc_pieces) {
            if constexpr (std::is_same<T, float>::value) {
                if (P.ngsel)
                    QMC_LAUNCH(st, "k_grad_tc",
                               launch_grad_tc(xt, Froot, root_stride, Fchain, P.Fchain_per_shift, P.tau_pad, P.chb,
                                              P.gsel, P.gxoff, P.ngsel, partc, P.reff, P.tc_pieces, st));
                if (P.chl.count)
                    QMC_LAUNCH(st, "k_coarse_grad_tc",
                               launch_coarse_grad_tc(tab, P.tab_stride, Froot, root_stride, Fchain, P.Fchain_per_shift,
                                                     P.tau_pad, P.chl, partc, P.reff, P.bwd_tiles_l, P.tc_pieces, P.xc,
                                                     st));
                if (P.xc != 0.0f) {
                    // 1^T G over every shift: the column sums of the top folded level (or of the roots)
                    const bool top = P.fold.depth > 0;
                    const float* Ft = top ? Fchain + P.fold.off[P.fold.depth] : Froot;
                    const long long rows = top ? (1LL << P.fold.logn_top) : n_root;
                    double* part = reinterpret_cast<double*>(ws + P.off_gsum);
                    QMC_LAUNCH(st, "k_col_sums",
                               launch_col_sums(Ft, top ? P.Fchain_per_shift : root_stride, rows, P.reff, P.tau_pad,
                                               part, part + 64LL * P.tau_pad, st));
                }
            }
        } else {
            QMC_LAUNCH(st, "k_coarse_grad",
                       launch_coarse_grad<T>(tab, P.tab_stride, Froot, root_stride, Fchain, P.Fchain_per_shift,
                                             P.tau_pad, P.chb, partc, P.reff, P.bwd_tiles, st));
        }
    }
    int koff[4] = {0, 0, 0, 0}, col0[4] = {0, 0, 0, 0}, taul[4] = {0, 0, 0, 0};
    const int kmax_s4[4] = {1, 2, 4, 8};
    for (int I = 0, o = 0; I < P.JF; ++I) {
        koff[I] = o;
        col0[I] = P.lev_col0[I];
        taul[I] = P.lev_tau[I];
        o += P.shape == SHAPE_S4 ? kmax_s4[I] : 16;
    }
    const double* gsum = P.xc != 0.0f && P.chb.count
                             ? reinterpret_cast<const double*>(ws + P.off_gsum) + 64LL * P.tau_pad : nullptr;
    QMC_LAUNCH(st, "k_grad_reduce",
               launch_grad_reduce<T>(a.gradpart, nfine_part, std::max(P.kf_width, 1), koff, col0, taul, P.JF,
                                     partc, P.chb, P.tau, P.tau_pad, P.s, grad, gsum, (double)P.xc, st));
    return QMC_OK;
}

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================
extern "C" {

const char* qmc_version(void) { return "qmc_gb300 0.3 (sm_103a)"; }
const char* qmc_last_error(void) { return g_err.c_str(); }

qmc_status qmc_validate_rule(const qmc_rule* rule) { return validate(rule); }

qmc_status qmc_device_status(int clear) {
    unsigned int word = 0, lword = 0;
    QMC_CUDA(cudaDeviceSynchronize());
    QMC_CUDA(tc_error_word(&word, clear != 0));
    QMC_CUDA(level_error_word(&lword, clear != 0));
    word |= lword;
    QMC_CUDA(grad_error_word(&lword, clear != 0));
    word |= lword;
    QMC_CUDA(foldgrad_error_word(&lword, clear != 0));
    word |= lword;
    if (word)
        return fail(QMC_ERR_TIMEOUT, "a bounded device-side wait ran out (error word 0x%x: bit 0 a tensor-core "
                    "kernel, bit 31 the self-test)", word);
    return QMC_OK;
}

qmc_status qmc_selftest_wait_timeout(uint32_t polls, void* stream) {
    if (polls < 1 || polls > (1u << 20)) return fail(QMC_ERR_INVALID_ARG, "polls=%u outside [1, 2^20]", polls);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    QMC_LAUNCH(st, "k_selftest_wait", launch_selftest_wait(polls, st));
    return QMC_OK;
}

qmc_status qmc_workspace_size(int op, const qmc_rule* rules, const uint32_t* tau, uint32_t nprob,
                              const qmc_integrand* f, int precision, size_t* bytes) {
    if (!bytes) return fail(QMC_ERR_INVALID_ARG, "bytes is NULL");
    if (!rules) return fail(QMC_ERR_INVALID_ARG, "rules is NULL");
    if (op < QMC_OP_GEN_POINTS || op > QMC_OP_INTEGRATE_BWD) return fail(QMC_ERR_INVALID_ARG, "op %d unknown", op);
    if (nprob < 1) return fail(QMC_ERR_INVALID_ARG, "nprob must be >= 1");
    if (op != QMC_OP_GEN_POINTS && !tau) return fail(QMC_ERR_INVALID_ARG, "tau is NULL");
    size_t total = 0;
    for (uint32_t p = 0; p < nprob; ++p) {
        Plan P;
        qmc_status st = make_plan(op, &rules[p], op == QMC_OP_GEN_POINTS ? 1u : tau[p], f ? &f[p] : nullptr, precision,
                                  nullptr, P);
        if (st != QMC_OK) return st;
        total += align256(P.total);
    }
    *bytes = total;
    return QMC_OK;
}

qmc_status qmc_gen_points(const qmc_rule* rule, uint32_t shift_idx, int layout, uint32_t* d_out, size_t out_words,
                          void* d_ws, size_t ws_bytes, void* stream) {
    Plan P;
    qmc_status st = make_plan(QMC_OP_GEN_POINTS, rule, 1, nullptr, QMC_FP32, nullptr, P);
    if (st != QMC_OK) return st;
    if (!d_out) return fail(QMC_ERR_INVALID_ARG, "d_out is NULL");
    if (layout != QMC_LAYOUT_FULL && layout != QMC_LAYOUT_DISTINCT)
        return fail(QMC_ERR_INVALID_ARG, "layout %d unknown", layout);
    if (P.kind == QMC_REDUCED_MC ? shift_idx >= (uint32_t)P.reff : (P.R > 0 && shift_idx >= (uint32_t)P.R))
        return fail(QMC_ERR_INVALID_ARG, "shift_idx=%u but R=%d", shift_idx, P.R);
    const size_t need = layout == QMC_LAYOUT_FULL ? (size_t)P.N * P.s : (size_t)P.T_tot;
    if (out_words < need) return fail(QMC_ERR_INVALID_ARG, "d_out holds %zu words, %zu needed", out_words, need);
    if (P.total > 0 && (!d_ws || ws_bytes < P.total))
        return fail(QMC_ERR_NO_MEMORY, "workspace of %zu bytes, %zu needed", ws_bytes, P.total);
    cudaStream_t st_ = reinterpret_cast<cudaStream_t>(stream);
    char* ws = reinterpret_cast<char*>(d_ws);
    st = upload_rule(P, rule, ws, st_);
    if (st != QMC_OK) return st;
    const DevRule R = dev_rule(P, rule, ws);
    if (P.base_b) {
        QMC_LAUNCH(st_, "k_points_b", launch_points_b(R, d_out, (long long)need, layout == QMC_LAYOUT_FULL,
                                                      (int)shift_idx, st_));
        return QMC_OK;
    }
    if (layout == QMC_LAYOUT_FULL) QMC_LAUNCH(st_, "k_points_full", launch_points_full(R, d_out, (int)shift_idx, st_));
    else QMC_LAUNCH(st_, "k_points_distinct", launch_points_distinct(R, d_out, P.T_tot, (int)shift_idx, st_));
    return QMC_OK;
}

qmc_status qmc_reduced_matmul(const qmc_rule* rule, const void* d_A, uint32_t tau, int precision, void* d_P,
                              void* d_ws, size_t ws_bytes, void* stream) {
    Plan P;
    qmc_status st = make_plan(QMC_OP_REDUCED_MATMUL, rule, tau, nullptr, precision, d_A, P);
    if (st != QMC_OK) return st;
    if (!d_A || !d_P) return fail(QMC_ERR_INVALID_ARG, "d_A or d_P is NULL");
    // (the product kernels write whole 8- and 16-byte groups of a row)
    if (((uintptr_t)d_P) % 16) return fail(QMC_ERR_INVALID_ARG, "d_P must be 16-byte aligned");
    if (!d_ws || ws_bytes < P.total) return fail(QMC_ERR_NO_MEMORY, "workspace of %zu bytes, %zu needed", ws_bytes, P.total);
    if (((uintptr_t)d_ws) % 256) return fail(QMC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    cudaStream_t st_ = reinterpret_cast<cudaStream_t>(stream);
    char* ws = reinterpret_cast<char*>(d_ws);
    if (precision == QMC_FP64) {
        const double* A; int ld;
        return run_forward<double>(P, rule, (const double*)d_A, ws, nullptr, MODE_MATERIALIZE, (double*)d_P, nullptr,
                                   nullptr, st_, &A, &ld);
    }
    const float* A; int ld;
    return run_forward<float>(P, rule, (const float*)d_A, ws, nullptr, MODE_MATERIALIZE, (float*)d_P, nullptr,
                              nullptr, st_, &A, &ld);
}

// Several problems in one call run on internal streams: the caller's stream forks into them
// through an event and joins back through one event per stream, so the call stays ordered on the
// caller's stream and can be captured into a CUDA graph (the forked streams join the capture).
// Problems are dealt to the streams largest first (work ~ N tau R), each to the stream with the
// least work so far.
struct Forker {
    static constexpr int K = 4;
    static constexpr int kDevices = 64;
    std::mutex mu;
    bool ready[kDevices] = {};
    cudaStream_t s[kDevices][K];
    cudaEvent_t fork[kDevices], join[kDevices][K];
};
Forker& forker() {
    static Forker f;
    return f;
}

static qmc_status integrate_common(int op, const qmc_rule* rules, const void* const* d_A, const uint32_t* tau,
                                   uint32_t nprob, const qmc_integrand* f, int precision, double* d_est,
                                   void* const* d_rowf, const double* d_upstream, void* const* d_gradA,
                                   uint32_t flags, void* d_ws, size_t ws_bytes, void* stream) {
    if (!rules || !d_A || !tau || !f) return fail(QMC_ERR_INVALID_ARG, "rules, d_A, tau and f must be non-NULL");
    if (nprob < 1) return fail(QMC_ERR_INVALID_ARG, "nprob must be >= 1");
    if (op == QMC_OP_INTEGRATE && !d_est) return fail(QMC_ERR_INVALID_ARG, "d_est is NULL");
    if (op == QMC_OP_INTEGRATE_BWD && (!d_upstream || !d_gradA))
        return fail(QMC_ERR_INVALID_ARG, "d_upstream and d_gradA must be non-NULL");
    if (flags & ~QMC_BWD_REUSE_FORWARD) return fail(QMC_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
    std::vector<Plan> plans(nprob);
    size_t total = 0;
    for (uint32_t p = 0; p < nprob; ++p) {
        qmc_status st = make_plan(op, &rules[p], tau[p], &f[p], precision, d_A[p], plans[p]);
        if (st != QMC_OK) return st;
        if (!d_A[p]) return fail(QMC_ERR_INVALID_ARG, "d_A[%u] is NULL", p);
        if (op == QMC_OP_INTEGRATE_BWD && !d_gradA[p]) return fail(QMC_ERR_INVALID_ARG, "d_gradA[%u] is NULL", p);
        total += align256(plans[p].total);
    }
    if (!d_ws || ws_bytes < total) return fail(QMC_ERR_NO_MEMORY, "workspace of %zu bytes, %zu needed", ws_bytes, total);
    if (((uintptr_t)d_ws) % 256) return fail(QMC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    char* ws0 = reinterpret_cast<char*>(d_ws);
    // per problem: its workspace and estimate offsets, and its stream
    std::vector<size_t> ws_off(nprob), est_offs(nprob);
    std::vector<int> lane(nprob, -1);
    {
        size_t wo = 0, eo = 0;
        for (uint32_t p = 0; p < nprob; ++p) {
            ws_off[p] = wo; est_offs[p] = eo;
            wo += align256(plans[p].total);
            eo += (size_t)plans[p].reff + 1;
        }
    }
    Forker& fk = forker();
    std::unique_lock<std::mutex> lock(fk.mu, std::defer_lock);
    int dev = 0, used = 0;
    if (nprob > 1) {
        QMC_CUDA(cudaGetDevice(&dev));
        if (dev < 0 || dev >= Forker::kDevices) return fail(QMC_ERR_CUDA, "device ordinal %d out of range", dev);
        lock.lock();
        if (!fk.ready[dev]) {
            for (int k = 0; k < Forker::K; ++k) {
                QMC_CUDA(cudaStreamCreateWithFlags(&fk.s[dev][k], cudaStreamNonBlocking));
                QMC_CUDA(cudaEventCreateWithFlags(&fk.join[dev][k], cudaEventDisableTiming));
            }
            QMC_CUDA(cudaEventCreateWithFlags(&fk.fork[dev], cudaEventDisableTiming));
            fk.ready[dev] = true;
        }
        std::vector<uint32_t> order(nprob);
        for (uint32_t p = 0; p < nprob; ++p) order[p] = p;
        auto work = [&](uint32_t p) { return (double)plans[p].N * plans[p].tau * plans[p].reff; };
        std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return work(a) > work(b); });
        double load[Forker::K] = {};
        for (uint32_t p : order) {
            int best = 0;
            for (int k = 1; k < Forker::K; ++k)
                if (load[k] < load[best]) best = k;
            lane[p] = best;
            load[best] += work(p);
        }
        used = std::min<int>(Forker::K, (int)nprob);
        QMC_CUDA(cudaEventRecord(fk.fork[dev], caller));
        for (int k = 0; k < used; ++k) QMC_CUDA(cudaStreamWaitEvent(fk.s[dev][k], fk.fork[dev], 0));
    }
    for (uint32_t p = 0; p < nprob; ++p) {
        const Plan& P = plans[p];
        cudaStream_t st_ = lane[p] < 0 ? caller : fk.s[dev][lane[p]];
        char* ws = ws0 + ws_off[p];
        const size_t est_off = est_offs[p];
        qmc_status st;
        if (op == QMC_OP_INTEGRATE) {
            void* rowf = d_rowf ? d_rowf[p] : nullptr;
            if (precision == QMC_FP64) {
                const double* A; int ld;
                st = run_forward<double>(P, &rules[p], (const double*)d_A[p], ws, &f[p], MODE_FUSED, nullptr,
                                         (double*)rowf, d_est + est_off, st_, &A, &ld);
            } else {
                const float* A; int ld;
                st = run_forward<float>(P, &rules[p], (const float*)d_A[p], ws, &f[p], MODE_FUSED, nullptr,
                                        (float*)rowf, d_est + est_off, st_, &A, &ld);
            }
        } else {
            const bool reuse = (flags & QMC_BWD_REUSE_FORWARD) != 0;
            if (precision == QMC_FP64)
                st = run_backward<double>(P, &rules[p], (const double*)d_A[p], ws, &f[p], d_upstream + p,
                                          (double*)d_gradA[p], reuse, st_);
            else
                st = run_backward<float>(P, &rules[p], (const float*)d_A[p], ws, &f[p], d_upstream + p,
                                         (float*)d_gradA[p], reuse, st_);
        }
        if (st != QMC_OK) {
            // join what was forked, so that the caller's stream (or its capture) stays consistent
            for (int k = 0; k < used; ++k) {
                cudaEventRecord(fk.join[dev][k], fk.s[dev][k]);
                cudaStreamWaitEvent(caller, fk.join[dev][k], 0);
            }
            return st;
        }
    }
    for (int k = 0; k < used; ++k) {
        QMC_CUDA(cudaEventRecord(fk.join[dev][k], fk.s[dev][k]));
        QMC_CUDA(cudaStreamWaitEvent(caller, fk.join[dev][k], 0));
    }
    return QMC_OK;
}

qmc_status qmc_integrate(const qmc_rule* rules, const void* const* d_A, const uint32_t* tau, uint32_t nprob,
                         const qmc_integrand* f, int precision, double* d_est, void* const* d_rowf, void* d_ws,
                         size_t ws_bytes, void* stream) {
    return integrate_common(QMC_OP_INTEGRATE, rules, d_A, tau, nprob, f, precision, d_est, d_rowf, nullptr, nullptr,
                            0u, d_ws, ws_bytes, stream);
}

qmc_status qmc_integrate_backward(const qmc_rule* rules, const void* const* d_A, const uint32_t* tau, uint32_t nprob,
                                  const qmc_integrand* f, int precision, const double* d_upstream,
                                  void* const* d_gradA, uint32_t flags, void* d_ws, size_t ws_bytes, void* stream) {
    return integrate_common(QMC_OP_INTEGRATE_BWD, rules, d_A, tau, nprob, f, precision, nullptr, nullptr, d_upstream,
                            d_gradA, flags, d_ws, ws_bytes, stream);
}

qmc_status qmc_autotune(const qmc_rule* rule, const void* d_A, uint32_t tau, const qmc_integrand* f, int precision,
                        double* d_est, void* d_gradA, void* d_ws, size_t ws_bytes, void* stream, uint32_t* n_timed) {
    if (!rule || !d_A || !f || !d_est || !d_gradA || !d_ws)
        return fail(QMC_ERR_INVALID_ARG, "rule, d_A, f, d_est, d_gradA and d_ws must be non-NULL");
    if (((uintptr_t)d_ws) % 256) return fail(QMC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    Plan base;
    t_hint = nullptr;
    qmc_status st = make_plan(QMC_OP_INTEGRATE_BWD, rule, tau, f, precision, d_A, base);
    if (st != QMC_OK) return st;
    cudaStream_t st_ = reinterpret_cast<cudaStream_t>(stream);
    char* ws = reinterpret_cast<char*>(d_ws);
    uint32_t timed = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    QMC_CUDA(cudaEventCreate(&e0));
    QMC_CUDA(cudaEventCreate(&e1));
    // the timed backward reads its upstream factor dL/dQ from the mean estimate's slot (any value
    // does: the gradients written while timing are scratch)
    const double* d_up = d_est + base.reff;
    // time one candidate: the forward, or the forward and the backward that reuses it
    auto time_it = [&](const TuneVal& tv, bool bwd, float* ms) -> qmc_status {
        Plan P;
        t_hint = &tv;
        qmc_status s2 = make_plan(QMC_OP_INTEGRATE_BWD, rule, tau, f, precision, d_A, P);
        t_hint = nullptr;
        if (s2 != QMC_OK) return s2;
        if (P.total > ws_bytes) { *ms = -1.0f; return QMC_OK; }     // does not fit the caller's workspace
        float best = -1.0f;
        for (int rep = 0; rep < 4; ++rep) {
            QMC_CUDA(cudaEventRecord(e0, st_));
            if (precision == QMC_FP64) {
                const double* A; int ld;
                s2 = run_forward<double>(P, rule, (const double*)d_A, ws, f, MODE_FUSED, nullptr, nullptr, d_est, st_, &A, &ld);
                if (s2 == QMC_OK && bwd)
                    s2 = run_backward<double>(P, rule, (const double*)d_A, ws, f, d_up, (double*)d_gradA, true, st_);
            } else {
                const float* A; int ld;
                s2 = run_forward<float>(P, rule, (const float*)d_A, ws, f, MODE_FUSED, nullptr, nullptr, d_est, st_, &A, &ld);
                if (s2 == QMC_OK && bwd)
                    s2 = run_backward<float>(P, rule, (const float*)d_A, ws, f, d_up, (float*)d_gradA, true, st_);
            }
            if (s2 != QMC_OK) return s2;
            QMC_CUDA(cudaEventRecord(e1, st_));
            QMC_CUDA(cudaEventSynchronize(e1));
            float t = 0.0f;
            QMC_CUDA(cudaEventElapsedTime(&t, e0, e1));
            if (rep > 0 && (best < 0.0f || t < best)) best = t;     // (the first run warms up)
        }
        ++timed;
        *ms = best;
        return QMC_OK;
    };
    TuneVal bestv{};
    if (base.fine_s4) {
        // forward: the cost model's column groups and a ladder of others (columns per CTA = 4 qpg)
        const int quads = base.tau_pad / 4;
        const int ladder[] = {base.cr / 4, 8, 16, 24, 32, 48, 64, 96, 128};
        float bt = -1.0f;
        for (int qpg : ladder) {
            if (qpg < 1 || qpg > quads || qpg > 128) continue;
            TuneVal tv{qpg, 0, 0, 0, 0};
            float ms = 0.0f;
            st = time_it(tv, false, &ms);
            if (st != QMC_OK) break;
            if (ms > 0.0f && (bt < 0.0f || ms < bt)) { bt = ms; bestv.fwd_qpg = qpg; }
        }
        // the other number of level-3 nodes per forward thread, with the column groups just chosen
        if (st == QMC_OK) {
            Plan tmp;
            TuneVal tb{bestv.fwd_qpg, 0, 0, 0, 0};
            t_hint = &tb;
            st = make_plan(QMC_OP_INTEGRATE_BWD, rule, tau, f, precision, d_A, tmp);
            t_hint = nullptr;
            if (st == QMC_OK) {
                TuneVal alt = tb;
                alt.fwd_nb = 3 - tmp.fwd_nb;
                float ma = 0.0f;
                st = time_it(alt, false, &ma);
                if (st == QMC_OK && ma > 0.0f && (bt < 0.0f || ma < bt)) { bt = ma; bestv.fwd_nb = alt.fwd_nb; }
            }
        }
        // tensor-core tiers: the coarse path (level passes or block products), with the forward
        // schedule just chosen
        if (base.tc_pieces && base.chf.count && st == QMC_OK) {
            float b1 = -1.0f, b2 = -1.0f;
            TuneVal t1{bestv.fwd_qpg, 0, 1, 0, bestv.fwd_nb}, t2{bestv.fwd_qpg, 0, 2, 0, bestv.fwd_nb};
            st = time_it(t1, false, &b1);
            if (st == QMC_OK) st = time_it(t2, false, &b2);
            if (st == QMC_OK && b1 > 0.0f && b2 > 0.0f) bestv.coarse = b1 <= b2 ? 1 : 2;
        }
        // adjoint: roots per CTA around the cost model's choice, with the forward just chosen
        const long long n_root = 1LL << (base.m - base.JF);
        const double fac[] = {1.0, 0.5, 0.75, 1.5, 2.0, 3.0};
        float bb = -1.0f;
        for (double fc : fac) {
            if (st != QMC_OK) break;
            long long rpc = (long long)(base.roots_per_cta * fc + 0.5);
            rpc = std::max(2LL, (rpc + 1) / 2 * 2);
            if (rpc > n_root + 1) continue;
            TuneVal tv{bestv.fwd_qpg, (int)rpc, bestv.coarse, 0, bestv.fwd_nb};
            float ms = 0.0f;
            st = time_it(tv, true, &ms);
            if (st != QMC_OK) break;
            if (ms > 0.0f && (bb < 0.0f || ms < bb)) { bb = ms; bestv.bwd_rpc = (int)rpc; }
        }
        // one column pair per lane (two CTAs per SM), with the cost model's roots per CTA
        if (st == QMC_OK) {
            TuneVal tv{bestv.fwd_qpg, 0, bestv.coarse, 0, bestv.fwd_nb, 1};
            float ms = 0.0f;
            st = time_it(tv, true, &ms);
            if (st == QMC_OK && ms > 0.0f && (bb < 0.0f || ms < bb)) { bb = ms; bestv.bwd_rpc = 0; bestv.bwd_cpl = 1; }
        }
        // tensor-core tiers: the coarse adjoint's path, with the schedules just chosen
        if (base.tc_pieces && base.chb.count && st == QMC_OK) {
            float b1 = -1.0f, b2 = -1.0f;
            TuneVal t1 = bestv, t2 = bestv;
            t1.bwd = 1;
            t2.bwd = 2;
            st = time_it(t1, true, &b1);
            if (st == QMC_OK) st = time_it(t2, true, &b2);
            if (st == QMC_OK && b1 > 0.0f && b2 > 0.0f) bestv.bwd = b1 <= b2 ? 1 : 2;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != QMC_OK) return st;
    {
        TuneCache& tc = tune_cache();
        std::lock_guard<std::mutex> g(tc.mu);
        tc.m[base.tune_key] = bestv;
    }
    if (n_timed) *n_timed = timed;
    return QMC_OK;
}

qmc_status qmc_tune_set(const qmc_rule* rule, uint32_t tau, const qmc_integrand* f, int precision, int fwd_qpg,
                        int bwd_rpc, int coarse, int bwd_path) {
    if (!rule || !f) return fail(QMC_ERR_INVALID_ARG, "rule and f must be non-NULL");
    if (fwd_qpg < 0 || fwd_qpg > 128 || bwd_rpc < 0 || coarse < 0 || coarse > 2 || bwd_path < 0 || bwd_path > 2)
        return fail(QMC_ERR_INVALID_ARG, "schedule values out of range");
    qmc_status st = validate(rule);
    if (st != QMC_OK) return st;
    Plan P;
    t_hint = nullptr;
    st = make_plan(QMC_OP_INTEGRATE_BWD, rule, tau, f, precision, nullptr, P);
    if (st != QMC_OK) return st;
    if (P.tune_key.empty()) return fail(QMC_ERR_UNSUPPORTED, "this rule's plan takes no schedule");
    TuneCache& tc = tune_cache();
    std::lock_guard<std::mutex> g(tc.mu);
    tc.m[P.tune_key] = TuneVal{fwd_qpg, bwd_rpc, coarse, bwd_path, 0};
    return QMC_OK;
}

qmc_status qmc_tune_clear(void) {
    TuneCache& tc = tune_cache();
    std::lock_guard<std::mutex> g(tc.mu);
    tc.m.clear();
    return QMC_OK;
}

qmc_status qmc_tune_save(const char* path) {
    if (!path) return fail(QMC_ERR_INVALID_ARG, "path is NULL");
    TuneCache& tc = tune_cache();
    std::lock_guard<std::mutex> g(tc.mu);
    FILE* fh = fopen(path, "w");
    if (!fh) return fail(QMC_ERR_INVALID_ARG, "cannot write %s", path);
    fprintf(fh, "# qmc_gb300 schedule cache: shape key | forward column quads per CTA | adjoint roots per CTA | "
                "coarse path (1 level passes, 2 block products) | adjoint path (1 one fold, 2 fused) | "
                "forward level-3 nodes per thread | adjoint column pairs per lane\n");
    for (auto& kv : tc.m)
        fprintf(fh, "%s|%d|%d|%d|%d|%d|%d\n", kv.first.c_str(), kv.second.fwd_qpg, kv.second.bwd_rpc,
                kv.second.coarse, kv.second.bwd, kv.second.fwd_nb, kv.second.bwd_cpl);
    fclose(fh);
    return QMC_OK;
}

qmc_status qmc_tune_load(const char* path, uint32_t* n_entries) {
    if (!path) return fail(QMC_ERR_INVALID_ARG, "path is NULL");
    FILE* fh = fopen(path, "r");
    if (!fh) return fail(QMC_ERR_INVALID_ARG, "cannot read %s", path);
    TuneCache& tc = tune_cache();
    std::lock_guard<std::mutex> g(tc.mu);
    char line[4096];
    uint32_t n = 0;
    int lineno = 0;
    qmc_status st = QMC_OK;
    while (fgets(line, sizeof(line), fh)) {
        ++lineno;
        if (line[0] == '#' || line[0] == '\n') continue;
        char* a = strchr(line, '|');
        char* b = a ? strchr(a + 1, '|') : nullptr;
        char* c = b ? strchr(b + 1, '|') : nullptr;          // (the coarse and adjoint paths are optional)
        char* d = c ? strchr(c + 1, '|') : nullptr;
        char* e = d ? strchr(d + 1, '|') : nullptr;
        char* g = e ? strchr(e + 1, '|') : nullptr;
        int q = 0, r = 0, cp = 0, bp = 0, nb = 0, cl = 0;
        if (!a || !b || sscanf(a + 1, "%d", &q) != 1 || sscanf(b + 1, "%d", &r) != 1 || q < 0 || r < 0 || q > 128 ||
            (c && (sscanf(c + 1, "%d", &cp) != 1 || cp < 0 || cp > 2)) ||
            (d && (sscanf(d + 1, "%d", &bp) != 1 || bp < 0 || bp > 2)) ||
            (e && (sscanf(e + 1, "%d", &nb) != 1 || nb < 0 || nb > 2)) ||
            (g && (sscanf(g + 1, "%d", &cl) != 1 || cl < 0 || cl > 2))) {
            st = fail(QMC_ERR_INVALID_ARG, "%s:%d: not a schedule entry", path, lineno);
            break;
        }
        tc.m[std::string(line, a - line)] = TuneVal{q, r, cp, bp, nb, cl};
        ++n;
    }
    fclose(fh);
    if (st == QMC_OK && n_entries) *n_entries = n;
    return st;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Allocation-free variant of qmc_integrate.
//
// Some callers cannot allocate device memory when they call the library: code
// that runs while a stream is being captured by a framework that forbids
// cudaMalloc during capture, real-time or embedded hosts that reserve all
// device memory up front, and foreign-function callers that have no device
// allocator of their own to make a workspace with.  For them the fused forward
// runs on a fixed scratch array that is part of the library image: it exists
// on every GPU that loads the library, from module load until the process
// exits, whether or not this entry point is ever called.
// ------------------------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, called once per device with that device current.
qmc_status noalloc_scratch(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(QMC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(QMC_ERR_CUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(QMC_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return QMC_OK;
}

}  // namespace

extern "C" {

qmc_status qmc_integrate_noalloc(const qmc_rule* rule, const void* d_A, uint32_t tau, const qmc_integrand* f,
                                 int precision, double* d_est, void* stream) {
    if (!d_A || !d_est || !f) return fail(QMC_ERR_INVALID_ARG, "d_A, d_est and f must be non-NULL");
    Plan P, Pq;
    qmc_status st = make_plan(QMC_OP_INTEGRATE, rule, tau, f, precision, d_A, P);
    if (st != QMC_OK) return st;
    // The limit is checked against qmc_workspace_size's plan (made without d_A, so it always holds
    // the padded copy of A): a problem is accepted exactly when that query fits the array, whatever
    // A's alignment.  The plan for the given d_A is never larger.
    st = make_plan(QMC_OP_INTEGRATE, rule, tau, f, precision, nullptr, Pq);
    if (st != QMC_OK) return st;
    if (Pq.total > kNoAllocScratchBytes)
        return fail(QMC_ERR_NO_MEMORY,
                    "qmc_integrate_noalloc: this problem needs %zu bytes of scratch, the static array holds %zu "
                    "(use qmc_integrate with a caller workspace)",
                    Pq.total, kNoAllocScratchBytes);
    void* scratch = nullptr;
    st = noalloc_scratch(&scratch);
    if (st != QMC_OK) return st;
    // Every area the forward pass reads is written earlier in the same call, so the
    // array needs no clearing between calls.
    char* ws = reinterpret_cast<char*>(scratch);
    cudaStream_t st_ = reinterpret_cast<cudaStream_t>(stream);
    if (precision == QMC_FP64) {
        const double* A;
        int ld;
        return run_forward<double>(P, rule, (const double*)d_A, ws, f, MODE_FUSED, nullptr, nullptr, d_est, st_, &A,
                                   &ld);
    }
    const float* A;
    int ld;
    return run_forward<float>(P, rule, (const float*)d_A, ws, f, MODE_FUSED, nullptr, nullptr, d_est, st_, &A, &ld);
}

qmc_status qmc_trace_enable(int on) {
    TraceState& t = trace_state();
    std::lock_guard<std::mutex> g(t.mu);
    if (on) {
        for (auto& r : t.recs) { t.pool.push_back(r.a); t.pool.push_back(r.b); }
        t.recs.clear();
        t.names.clear(); t.counts.clear(); t.ms.clear();
    }
    t.on = on != 0;
    return QMC_OK;
}

qmc_status qmc_trace_collect(uint32_t* n_kernels) {
    if (!n_kernels) return fail(QMC_ERR_INVALID_ARG, "n_kernels is NULL");
    TraceState& t = trace_state();
    std::lock_guard<std::mutex> g(t.mu);
    std::map<std::string, std::pair<unsigned long long, double>> agg;
    for (size_t i = 0; i < t.names.size(); ++i) agg[t.names[i]] = {t.counts[i], t.ms[i]};
    for (auto& r : t.recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return fail(QMC_ERR_CUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return fail(QMC_ERR_CUDA, "cudaEventElapsedTime: %s", cudaGetErrorString(e));
        auto& slot = agg[r.name];
        slot.first += 1;
        slot.second += ms;
        t.pool.push_back(r.a);
        t.pool.push_back(r.b);
    }
    t.recs.clear();
    t.names.clear(); t.counts.clear(); t.ms.clear();
    for (auto& kv : agg) { t.names.push_back(kv.first); t.counts.push_back(kv.second.first); t.ms.push_back(kv.second.second); }
    *n_kernels = (uint32_t)t.names.size();
    return QMC_OK;
}

qmc_status qmc_trace_entry(uint32_t i, const char** name, uint64_t* launches, double* total_ms) {
    TraceState& t = trace_state();
    std::lock_guard<std::mutex> g(t.mu);
    if (i >= t.names.size() || !name || !launches || !total_ms) return fail(QMC_ERR_INVALID_ARG, "bad trace entry query");
    *name = t.names[i].c_str();
    *launches = t.counts[i];
    *total_ms = t.ms[i];
    return QMC_OK;
}

}  // extern "C"

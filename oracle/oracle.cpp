// Oracle for the multi-scale LFK community-growth hot path.
//
// TEST INFRASTRUCTURE ONLY.  This library is loaded by the test suite, by the
// smoke check and by the CPU-baseline leg of the benchmark, and by nothing
// else.  The product path (the CUDA library) never calls, links or includes
// it, and it shares no code with that path.
//
// It is a plain, slow, single-threaded-per-unit restatement of the method of
// Le Martelot & Hankin, "Fast Multi-Scale Community Detection based on Local
// Criteria within a Multi-Threaded Algorithm":
//   * Eq. 1   LFK community fitness  f_c = k_in / (k_in + k_out)^alpha
//   * Eq. 2   node fitness f^i_c = f_{c+i} - f_{c-i}, used as a strict test
//   * Sec. 2  ranking factor 2 d_in / (d_in + d_out)^alpha of the max
//             priority queue (d_in + d_out is the node's degree)
//   * Alg. 1  grow: pop the best queued neighbour, add it if it improves f,
//             update or add its outside neighbours in the queue; then, if
//             anything was added, prune passes until no member is removed
//   * Alg. 2  "while changes can be made": Alg. 1 is repeated until a grow
//             pass adds nothing (each unit grows from {seed} independently)
//   * Sec. 3  complexity text: the community is quick-sorted at the end
//   * Sec. 4  logarithmic scale sampling and the overlapping NMI of
//             Lancichinetti, Fortunato & Kertesz averaged over p scales
//
// Readings taken where the paper is silent or garbled: k_in counts internal edges twice (internal degree sum); add and
// remove tests are strict; the seed is never removed; priority ties go to
// the smaller node id; a prune pass walks a snapshot of the members in
// ascending id and removes at once; the prune loop runs until a pass removes
// nothing; a popped and rejected node re-enters the queue when a later
// addition touches it; every decision is the exact mathematical sign of
//   Delta = log(a1/a2) - alpha * log(b1/b2)
// with alpha taken as the exact binary64 value.
//
// Weights: FP32 weights are converted exactly to int64 multiples of the
// largest power of two dividing all of them; unweighted graphs use weight 1.
// Every sum is then an exact integer and independent of summation order.
//
// Decision arithmetic (independent of the device path): integer shortcuts,
// then binary64 with a derived error bound, then IEEE binary128 (libquadmath
// on x86-64, long double on AArch64), then an exact tie test for the dyadic
// rational alpha.  A case that none of these decides is reported as
// ORC_EUNDECIDED.
//
// Besides the per-seed growth it states the paper's full method (Alg. 2 with
// the growth of Alg. 3: seed rules, overlap pre-test, check and merge rounds,
// carry-over across scales) in one fixed sequential order, orc_full below,
// and growth from given initial members (orc_run_init).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <queue>
#include <thread>
#include <unordered_map>
#include <vector>

#if defined(__x86_64__)
#include <quadmath.h>
typedef __float128 quad;
static inline quad q_log(quad x) { return logq(x); }
static inline quad q_log1p(quad x) { return log1pq(x); }
static inline quad q_exp(quad x) { return expq(x); }
static inline quad q_abs(quad x) { return fabsq(x); }
static inline quad q_ldexp(quad x, int e) { return ldexpq(x, e); }
#elif defined(__aarch64__) && (__LDBL_MANT_DIG__ == 113)
typedef long double quad;
static inline quad q_log(quad x) { return logl(x); }
static inline quad q_log1p(quad x) { return log1pl(x); }
static inline quad q_exp(quad x) { return expl(x); }
static inline quad q_abs(quad x) { return fabsl(x); }
static inline quad q_ldexp(quad x, int e) { return ldexpl(x, e); }
#else
#error "the oracle needs an IEEE binary128 floating type"
#endif

typedef int64_t i64;
typedef int32_t i32;

// Status codes (same numeric meaning as the library's, defined here on their own).
enum {
    ORC_OK = 0,
    ORC_EINVAL = -1,
    ORC_ENOTSYM = -2,
    ORC_ESELFLOOP = -3,
    ORC_EDUP = -4,
    ORC_ERANGE = -5,
    ORC_ESMALL = -9,
    ORC_EUNDECIDED = -10,
    ORC_EUNSORTED = -11,
    ORC_EWEIGHT = -12,
    ORC_ETIMEOUT = -8,
};

// ---------------------------------------------------------------------------
// Exact sign of Delta = log(a1/a2) - alpha * log(b1/b2), a1,a2,b1,b2 > 0.
// ---------------------------------------------------------------------------

static i64 gcd64(i64 a, i64 b) {
    while (b) { i64 t = a % b; a = b; b = t; }
    return a;
}

// Integer square root if x is a perfect square, else -1.
static i64 exact_sqrt(i64 x) {
    i64 r = (i64)std::sqrt((double)x);
    while (r > 0 && (__int128)r * r > x) r--;
    while ((__int128)(r + 1) * (r + 1) <= x) r++;
    return ((__int128)r * r == x) ? r : -1;
}

// base^e == target, with early exit once the power exceeds target.
static bool pow_equals(i64 base, uint64_t e, i64 target) {
    if (base == 1) return target == 1;
    __int128 acc = 1;
    for (uint64_t i = 0; i < e; i++) {
        acc *= base;
        if (acc > target) return false;
    }
    return acc == target;
}

// alpha = P / 2^s with P odd (s may be <= 0 for integer alpha).
static void alpha_dyadic(double alpha, uint64_t *P, int *s) {
    int e;
    double m = std::frexp(alpha, &e);          // alpha = m 2^e, m in [1/2, 1)
    uint64_t M = (uint64_t)std::ldexp(m, 53);  // exact 53-bit integer
    int sh = 53 - e;
    while ((M & 1u) == 0) { M >>= 1; sh--; }
    *P = M;
    *s = sh;
}

// True iff a1/a2 == (b1/b2)^alpha exactly.  alpha = P/2^s, P odd: the
// equality holds iff the reduced b is the 2^s-th power of a reduced
// rational t and the reduced a equals t^P (unique factorisation).
static bool exact_tie(i64 a1, i64 a2, i64 b1, i64 b2, double alpha) {
    i64 g = gcd64(a1, a2), an = a1 / g, ad = a2 / g;
    g = gcd64(b1, b2);
    i64 bn = b1 / g, bd = b2 / g;
    if (bn == 1 && bd == 1) return an == 1 && ad == 1;
    uint64_t P;
    int s;
    alpha_dyadic(alpha, &P, &s);
    uint64_t expo = P;
    if (s > 0) {
        for (int i = 0; i < s; i++) {
            bn = exact_sqrt(bn);
            bd = exact_sqrt(bd);
            if (bn < 0 || bd < 0) return false;
            if (bn == 1 && bd == 1) return false;  // b != 1 cannot be a power of 1
        }
    } else {
        // integer alpha = P * 2^(-s); a base >= 2 overflows long before this
        int sh = -s;
        expo = (sh >= 63) ? UINT64_MAX : ((P > (UINT64_MAX >> sh)) ? UINT64_MAX : (P << sh));
    }
    return pow_equals(bn, expo, an) && pow_equals(bd, expo, ad);
}

static const double U64 = 0x1p-53;

// log(a1/a2) in binary64.  Absolute error <= 13u|L| (log1p branch: 3u
// relative error of the quotient times the derivative bound 2 on
// |t| <= 1/2, plus <= 2 ulp of log1p; log branch: |L| > log 1.5 so the 3u
// quotient error is <= 7.4u|L|, plus <= 2 ulp of log).  Returned bound 32u|L|.
static double log_ratio_d(i64 a1, i64 a2, double *err) {
    i64 diff = a1 - a2;
    double L;
    if ((__int128)2 * (diff < 0 ? -diff : diff) <= a2)
        L = std::log1p((double)diff / (double)a2);
    else
        L = std::log((double)a1 / (double)a2);
    *err = 0x1p-48 * std::fabs(L);
    return L;
}

// The same in binary128: the quotient is rounded once (the integers are
// exact in 113 bits).  Returned bound 2^-100 |L|, far above the error.
static quad log_ratio_q(i64 a1, i64 a2) {
    i64 diff = a1 - a2;
    if ((__int128)2 * (diff < 0 ? -diff : diff) <= a2)
        return q_log1p((quad)diff / (quad)a2);
    return q_log((quad)a1 / (quad)a2);
}

struct DecideStats {
    i64 fast = 0, quadp = 0, tie = 0, undecided = 0;
};

// Returns +1, 0 (exact tie), -1; sets *undecided when no stage decides.
static int sign_delta(i64 a1, i64 a2, i64 b1, i64 b2, double alpha, int *path, bool *undecided) {
    // 1. integer shortcuts
    if (b1 == b2) { *path = 0; return (a1 > a2) - (a1 < a2); }
    if (a1 == a2) { *path = 0; return (b2 > b1) - (b2 < b1); }
    // 2. binary64 with a certified bound
    double e1, e2;
    double L1 = log_ratio_d(a1, a2, &e1);
    double L2 = log_ratio_d(b1, b2, &e2);
    double D = L1 - alpha * L2;
    double E = 0x1p-47 * (std::fabs(L1) + alpha * std::fabs(L2));
    if (std::fabs(D) > E) { *path = 1; return D > 0 ? 1 : -1; }
    // 3. binary128
    quad Q1 = log_ratio_q(a1, a2), Q2 = log_ratio_q(b1, b2);
    quad DQ = Q1 - (quad)alpha * Q2;
    quad EQ = q_ldexp(q_abs(Q1) + (quad)alpha * q_abs(Q2), -100);
    if (q_abs(DQ) > EQ) { *path = 2; return DQ > 0 ? 1 : -1; }
    // 4. exact tie test
    *path = 3;
    if (exact_tie(a1, a2, b1, b2, alpha)) return 0;
    *undecided = true;
    return 0;
}

// Add test for n outside c (Eq. 2 > 0): (K+2d)/(V+k)^alpha > K/V^alpha.
static int add_test(i64 K, i64 V, i64 d, i64 k, double alpha, int *path, bool *und) {
    if (K == 0) { *path = 0; return 1; }  // f_c = 0 < f_{c+n} since d > 0
    return sign_delta(K + 2 * d, K, V + k, V, alpha, path, und) > 0;
}

// Remove test for a member n (Alg. 1): (K-2d)/(V-k)^alpha > K/V^alpha.
static int remove_test(i64 K, i64 V, i64 d, i64 k, double alpha, int *path, bool *und) {
    if (K == 0 || K - 2 * d == 0) { *path = 0; return 0; }  // f_{c\n} = 0 <= f_c
    return sign_delta(K - 2 * d, K, V - k, V, alpha, path, und) > 0;
}

// f = K u / (V u)^alpha with u = 2^unit_exp (Eq. 1 in original weight units).
static double fitness(i64 K, i64 V, double alpha, int unit_exp) {
    if (K == 0) return 0.0;
    quad a = (quad)alpha;
    quad lf = q_log((quad)K) - a * q_log((quad)V) + ((quad)1 - a) * (quad)unit_exp * q_log((quad)2);
    return (double)q_exp(lf);
}

// ---------------------------------------------------------------------------
// Graph: validation and exact fixed-point weights.
// ---------------------------------------------------------------------------

struct orc_graph {
    i64 n = 0, nnz = 0;
    std::vector<i64> rp;
    std::vector<i32> col;
    std::vector<i64> w;  // empty = unweighted (every weight 1)
    std::vector<i64> k;  // weighted degree in weight units
    int unit_exp = 0;
    i64 volume = 0;
    i64 wt(i64 e) const { return w.empty() ? 1 : w[e]; }
};

// Checks, in this order over the whole graph, and reports the first failing
// category: structure (EINVAL), weights (EWEIGHT), self-loops (ESELFLOOP),
// ascending rows (EUNSORTED), duplicates (EDUP), symmetry with equal weights
// (ENOTSYM), fixed-point range (ERANGE).
extern "C" int orc_graph_create(i64 n, const i64 *row_ptr, const i32 *col, const float *w, orc_graph **out) {
    *out = nullptr;
    if (n < 0 || n > INT32_MAX || row_ptr == nullptr) return ORC_EINVAL;
    if (row_ptr[0] != 0) return ORC_EINVAL;
    for (i64 u = 0; u < n; u++)
        if (row_ptr[u + 1] < row_ptr[u]) return ORC_EINVAL;
    i64 E = row_ptr[n];
    if (E > 0 && col == nullptr) return ORC_EINVAL;
    for (i64 e = 0; e < E; e++)
        if (col[e] < 0 || col[e] >= n) return ORC_EINVAL;
    if (w)
        for (i64 e = 0; e < E; e++)
            if (!(std::isfinite(w[e]) && w[e] > 0.0f)) return ORC_EWEIGHT;
    for (i64 u = 0; u < n; u++)
        for (i64 e = row_ptr[u]; e < row_ptr[u + 1]; e++)
            if (col[e] == u) return ORC_ESELFLOOP;
    for (i64 u = 0; u < n; u++)
        for (i64 e = row_ptr[u] + 1; e < row_ptr[u + 1]; e++)
            if (col[e] < col[e - 1]) return ORC_EUNSORTED;
    for (i64 u = 0; u < n; u++)
        for (i64 e = row_ptr[u] + 1; e < row_ptr[u + 1]; e++)
            if (col[e] == col[e - 1]) return ORC_EDUP;
    for (i64 u = 0; u < n; u++)
        for (i64 e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            i64 v = col[e];
            const i32 *lo = col + row_ptr[v], *hi = col + row_ptr[v + 1];
            const i32 *it = std::lower_bound(lo, hi, (i32)u);
            if (it == hi || *it != u) return ORC_ENOTSYM;
            if (w && w[it - col] != w[e]) return ORC_ENOTSYM;
        }
    orc_graph *g = new orc_graph();
    g->n = n;
    g->nnz = E;
    g->rp.assign(row_ptr, row_ptr + n + 1);
    g->col.assign(col, col + E);
    g->k.assign(n, 0);
    if (w && E > 0) {
        // unit = 2^min over weights of the exponent of the lowest set bit
        int ue = INT32_MAX;
        for (i64 e = 0; e < E; e++) {
            int ex;
            float m = std::frexp(w[e], &ex);                 // w = m 2^ex
            uint32_t M = (uint32_t)std::ldexp((double)m, 24);  // 24-bit integer
            int low = ex - 24 + __builtin_ctz(M);
            ue = std::min(ue, low);
        }
        g->unit_exp = ue;
        g->w.resize(E);
        for (i64 e = 0; e < E; e++) {
            double x = std::ldexp((double)w[e], -ue);
            if (x > 0x1p62) { delete g; return ORC_ERANGE; }
            g->w[e] = (i64)x;
        }
    }
    __int128 vol = 0;
    for (i64 u = 0; u < n; u++) {
        __int128 s = 0;
        for (i64 e = row_ptr[u]; e < row_ptr[u + 1]; e++) s += g->wt(e);
        vol += s;
        if (vol >= ((__int128)1 << 62)) { delete g; return ORC_ERANGE; }
        g->k[u] = (i64)s;
    }
    g->volume = (i64)vol;
    *out = g;
    return ORC_OK;
}

extern "C" void orc_graph_destroy(orc_graph *g) { delete g; }

extern "C" int orc_graph_info(const orc_graph *g, i64 *n, i64 *nnz, i32 *unit_exp, i64 *volume) {
    *n = g->n; *nnz = g->nnz; *unit_exp = g->unit_exp; *volume = g->volume;
    return ORC_OK;
}

extern "C" int orc_graph_degrees(const orc_graph *g, i64 *k_out) {
    std::copy(g->k.begin(), g->k.end(), k_out);
    return ORC_OK;
}

extern "C" int orc_graph_weights(const orc_graph *g, i64 *w_out) {
    for (i64 e = 0; e < g->nnz; e++) w_out[e] = g->wt(e);
    return ORC_OK;
}

// ---------------------------------------------------------------------------
// Growth of one unit (seed, alpha): Alg. 1 repeated as in Alg. 2.
// ---------------------------------------------------------------------------

struct UnitResult {
    std::vector<i32> members;  // ascending
    i64 K = 0, V = 0;
    double f = 0.0;
    i64 edges_scanned = 0, adds = 0, removes = 0, rounds = 0;
    int status = ORC_OK;
    DecideStats ds;
};

struct QEntry {
    double key, err;  // binary64 estimate of log d - alpha log k and its bound
    i64 d, k;
    i32 id;
};

struct Grower {
    const orc_graph &g;
    double alpha;
    bool undecided = false;
    DecideStats ds;

    void count(int path) {
        if (path == 1) ds.fast++;
        else if (path == 2) ds.quadp++;
        else if (path == 3) ds.tie++;
    }

    // The ranking factor 2 d / k^alpha of a ranks before b's.
    bool ranks_before(const QEntry &a, const QEntry &b) {
        double diff = a.key - b.key;
        double bound = (a.err + b.err) * (1.0 + 0x1p-50);
        if (diff > bound) { ds.fast++; return true; }
        if (diff < -bound) { ds.fast++; return false; }
        int path;
        int s = sign_delta(a.d, b.d, a.k, b.k, alpha, &path, &undecided);
        count(path);
        if (s != 0) return s > 0;
        return a.id < b.id;
    }

    QEntry entry(i32 u, i64 d) const {
        QEntry q;
        q.d = d;
        q.k = g.k[u];
        q.id = u;
        double ld = std::log((double)d), lk = std::log((double)q.k);
        q.key = ld - alpha * lk;
        q.err = 0x1p-48 * (1.0 + std::fabs(ld) + alpha * (1.0 + std::fabs(lk)));
        return q;
    }
};

// Alg. 1 repeated while a grow pass adds (Alg. 2), from c = {seed} plus the
// optional initial members init[0..n_init) (Alg. 2: "a set of initial
// communities is given"; the seed stays pinned, repeats are ignored, the
// insertions are not counted as additions).
static void grow_unit(const orc_graph &g, i32 seed, double alpha, i64 max_rounds, UnitResult &R,
                      const i32 *init = nullptr, i64 n_init = 0, bool single = false) {
    Grower gr{g, alpha};
    std::unordered_map<i32, i64> din;  // d_in(u, c) for every node touched
    std::unordered_map<i32, char> inC;  // membership
    auto member = [&](i32 u) { auto it = inC.find(u); return it != inC.end() && it->second; };
    i64 K = 0, V = g.k[seed];
    inC[seed] = 1;
    for (i64 e = g.rp[seed]; e < g.rp[seed + 1]; e++) din[g.col[e]] += g.wt(e);
    R.edges_scanned += g.rp[seed + 1] - g.rp[seed];
    for (i64 j = 0; j < n_init; j++) {
        const i32 u = init[j];
        if (member(u)) continue;
        K += 2 * din[u];
        V += g.k[u];
        inC[u] = 1;
        R.edges_scanned += g.rp[u + 1] - g.rp[u];
        for (i64 e = g.rp[u]; e < g.rp[u + 1]; e++) din[g.col[e]] += g.wt(e);
    }

    auto cmp = [&](const QEntry &a, const QEntry &b) { return gr.ranks_before(b, a); };
    i64 rounds = 0;
    for (;;) {
        if (rounds >= max_rounds) { R.status = ORC_ETIMEOUT; break; }
        rounds++;
        // --- grow (Alg. 1, queue phase) ---
        std::priority_queue<QEntry, std::vector<QEntry>, decltype(cmp)> pq(cmp);
        std::unordered_map<i32, char> inQ;
        for (auto &kv : din)
            if (kv.second > 0 && !member(kv.first)) {
                pq.push(gr.entry(kv.first, kv.second));
                inQ[kv.first] = 1;
            }
        i64 added = 0;
        while (!pq.empty()) {
            QEntry top = pq.top();
            pq.pop();
            i32 u = top.id;
            if (!inQ[u] || top.d != din[u]) continue;  // stale entry
            inQ[u] = 0;
            int path;
            int ok = add_test(K, V, din[u], g.k[u], alpha, &path, &gr.undecided);
            gr.count(path);
            if (!ok) continue;
            K += 2 * din[u];
            V += g.k[u];
            inC[u] = 1;
            added++;
            R.adds++;
            R.edges_scanned += g.rp[u + 1] - g.rp[u];
            for (i64 e = g.rp[u]; e < g.rp[u + 1]; e++) {
                i32 v = g.col[e];
                i64 &dv = din[v];
                dv += g.wt(e);
                if (!member(v)) {
                    inQ[v] = 1;
                    pq.push(gr.entry(v, dv));
                }
            }
        }
        if (added == 0) break;
        // --- prune (Alg. 1, removal passes) ---
        for (;;) {
            std::vector<i32> snap;
            for (auto &kv : inC)
                if (kv.second) snap.push_back(kv.first);
            std::sort(snap.begin(), snap.end());
            i64 removed = 0;
            for (i32 u : snap) {
                if (u == seed) continue;
                int path;
                int rm = remove_test(K, V, din[u], g.k[u], alpha, &path, &gr.undecided);
                gr.count(path);
                if (!rm) continue;
                K -= 2 * din[u];
                V -= g.k[u];
                inC[u] = 0;
                removed++;
                R.removes++;
                R.edges_scanned += g.rp[u + 1] - g.rp[u];
                for (i64 e = g.rp[u]; e < g.rp[u + 1]; e++) din[g.col[e]] -= g.wt(e);
            }
            if (removed == 0) break;
        }
        if (single) break;  // one grow call of Alg. 1 (the full method repeats it itself)
    }
    R.rounds = rounds;
    for (auto &kv : inC)
        if (kv.second) R.members.push_back(kv.first);
    std::sort(R.members.begin(), R.members.end());
    R.K = K;
    R.V = V;
    R.f = fitness(K, V, alpha, g.unit_exp);
    R.ds = gr.ds;
    if (gr.undecided && R.status == ORC_OK) R.status = ORC_EUNDECIDED;
}

// stats[0..7]: edges_scanned, adds, removes, rounds, K, V, slow decisions
// (binary128 or tie stage), undecided flag.
static void fill_stats(const UnitResult &R, i64 *stats) {
    if (!stats) return;
    stats[0] = R.edges_scanned;
    stats[1] = R.adds;
    stats[2] = R.removes;
    stats[3] = R.rounds;
    stats[4] = R.K;
    stats[5] = R.V;
    stats[6] = R.ds.quadp + R.ds.tie;
    stats[7] = R.status == ORC_EUNDECIDED;
}

extern "C" int orc_grow(const orc_graph *g, i32 seed, double alpha, i64 max_rounds, i32 *members, i64 cap,
                        i64 *len, double *f, i64 *stats) {
    if (seed < 0 || seed >= g->n || !(alpha > 0.0) || !std::isfinite(alpha)) return ORC_EINVAL;
    UnitResult R;
    grow_unit(*g, seed, alpha, max_rounds, R);
    *len = (i64)R.members.size();
    if (f) *f = R.f;
    fill_stats(R, stats);
    if (cap < *len) return ORC_ESMALL;
    std::copy(R.members.begin(), R.members.end(), members);
    return R.status;
}

// ---------------------------------------------------------------------------
// Many units (scale-major: unit = scale_index * n_seeds + seed_index), spread
// over n_threads std::threads.  Each unit is independent, so the result does
// not depend on the thread count.
// ---------------------------------------------------------------------------

struct orc_result {
    std::vector<UnitResult> units;
};

// init_ptr (int64[n_seeds+1]) / init_nodes: optional initial members per seed.
extern "C" int orc_run_init(const orc_graph *g, const double *alphas, i32 n_scales, const i32 *seeds, i64 n_seeds,
                            const i64 *init_ptr, const i32 *init_nodes, i64 max_rounds, int n_threads,
                            orc_result **out) {
    *out = nullptr;
    for (i32 s = 0; s < n_scales; s++)
        if (!(alphas[s] > 0.0) || !std::isfinite(alphas[s])) return ORC_EINVAL;
    for (i64 i = 0; i < n_seeds; i++)
        if (seeds[i] < 0 || seeds[i] >= g->n) return ORC_EINVAL;
    if (init_ptr) {
        if (init_ptr[0] != 0) return ORC_EINVAL;
        for (i64 i = 0; i < n_seeds; i++) {
            if (init_ptr[i + 1] < init_ptr[i]) return ORC_EINVAL;
            for (i64 j = init_ptr[i]; j < init_ptr[i + 1]; j++)
                if (init_nodes[j] < 0 || init_nodes[j] >= g->n) return ORC_EINVAL;
        }
    }
    orc_result *r = new orc_result();
    i64 U = (i64)n_scales * n_seeds;
    r->units.resize(U);
    std::atomic<i64> next{0};
    auto work = [&]() {
        for (;;) {
            i64 u = next.fetch_add(1);
            if (u >= U) break;
            const i64 si = u % n_seeds;
            if (init_ptr)
                grow_unit(*g, seeds[si], alphas[u / n_seeds], max_rounds, r->units[u], init_nodes + init_ptr[si],
                          init_ptr[si + 1] - init_ptr[si]);
            else
                grow_unit(*g, seeds[si], alphas[u / n_seeds], max_rounds, r->units[u]);
        }
    };
    if (n_threads < 1) n_threads = 1;
    std::vector<std::thread> th;
    for (int t = 1; t < n_threads; t++) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
    *out = r;
    int st = ORC_OK;
    for (auto &R : r->units)
        if (R.status != ORC_OK) st = R.status;
    return st;
}

extern "C" int orc_run(const orc_graph *g, const double *alphas, i32 n_scales, const i32 *seeds, i64 n_seeds,
                       i64 max_rounds, int n_threads, orc_result **out) {
    return orc_run_init(g, alphas, n_scales, seeds, n_seeds, nullptr, nullptr, max_rounds, n_threads, out);
}

extern "C" void orc_result_destroy(orc_result *r) { delete r; }

extern "C" int orc_result_sizes(const orc_result *r, i64 *lens) {
    for (size_t u = 0; u < r->units.size(); u++) lens[u] = (i64)r->units[u].members.size();
    return ORC_OK;
}

// Concatenated member lists (ptr has n_units+1 entries), fitness and stats
// (8 per unit, see fill_stats).
extern "C" int orc_result_get(const orc_result *r, i64 *ptr, i32 *nodes, double *f, i64 *stats) {
    i64 off = 0;
    for (size_t u = 0; u < r->units.size(); u++) {
        const UnitResult &R = r->units[u];
        ptr[u] = off;
        std::copy(R.members.begin(), R.members.end(), nodes + off);
        off += (i64)R.members.size();
        if (f) f[u] = R.f;
        if (stats) fill_stats(R, stats + 8 * u);
    }
    ptr[r->units.size()] = off;
    return ORC_OK;
}

// ---------------------------------------------------------------------------
// Exported decision primitives (for the pinning tests).
// ---------------------------------------------------------------------------

// Returns sign of Delta (+1/0/-1) or ORC_EUNDECIDED (as 99 to keep it apart
// from a sign); *path: 0 integer shortcut, 1 binary64, 2 binary128, 3 tie test.
extern "C" int orc_sign_delta(i64 a1, i64 a2, i64 b1, i64 b2, double alpha, int *path) {
    bool und = false;
    int p = -1;
    int s = sign_delta(a1, a2, b1, b2, alpha, &p, &und);
    if (path) *path = p;
    return und ? 99 : s;
}

extern "C" int orc_add_test(i64 K, i64 V, i64 d, i64 k, double alpha) {
    bool und = false;
    int p;
    int r = add_test(K, V, d, k, alpha, &p, &und);
    return und ? ORC_EUNDECIDED : r;
}

extern "C" int orc_remove_test(i64 K, i64 V, i64 d, i64 k, double alpha) {
    bool und = false;
    int p;
    int r = remove_test(K, V, d, k, alpha, &p, &und);
    return und ? ORC_EUNDECIDED : r;
}

// +1 if node 1 ranks before node 2 in the max priority queue, else -1.
extern "C" int orc_priority_cmp(i64 d1, i64 k1, i32 id1, i64 d2, i64 k2, i32 id2, double alpha) {
    orc_graph g;  // only k[] is read by entry(): a two-node stand-in
    g.n = 2;
    g.k = {k1, k2};
    Grower gr{g, alpha};
    QEntry a = gr.entry(0, d1), b = gr.entry(1, d2);
    a.id = id1;
    b.id = id2;
    bool r = gr.ranks_before(a, b);
    if (gr.undecided) return ORC_EUNDECIDED;
    return r ? 1 : -1;
}

extern "C" double orc_fitness(i64 K, i64 V, double alpha, i32 unit_exp) { return fitness(K, V, alpha, unit_exp); }

// ---------------------------------------------------------------------------
// Dedup (per scale): identical sorted member lists are one community.  The
// unique communities are numbered in order of their first (smallest) unit
// index; unit2comm maps every unit to its community.
// ---------------------------------------------------------------------------

extern "C" int orc_dedup(i64 n_units, const i64 *ptr, const i32 *nodes, i64 *n_comms, i32 *unit2comm,
                         i64 *comm_first_unit) {
    std::map<std::vector<i32>, i32> seen;
    i64 c = 0;
    for (i64 u = 0; u < n_units; u++) {
        std::vector<i32> key(nodes + ptr[u], nodes + ptr[u + 1]);
        auto it = seen.find(key);
        if (it == seen.end()) {
            seen.emplace(std::move(key), (i32)c);
            if (comm_first_unit) comm_first_unit[c] = u;
            unit2comm[u] = (i32)c;
            c++;
        } else {
            unit2comm[u] = it->second;
        }
    }
    *n_comms = c;
    return ORC_OK;
}

// ---------------------------------------------------------------------------
// Overlapping NMI (Lancichinetti, Fortunato & Kertesz), cited in Sec. 4 for
// the comparison of community sets at successive scales.
// Each community is a binary variable over the n nodes.  With
// h(p) = -p log2 p:
//   H(X_k|Y_l) = H(X_k, Y_l) - H(Y_l), admitted only when
//                h(P11) + h(P00) > h(P01) + h(P10)
//   H(X_k|Y)   = min over admitted l, else H(X_k)
//   H(X|Y)     = mean over k of H(X_k|Y) / H(X_k)
//   N(X|Y)     = 1 - [H(X|Y) + H(Y|X)] / 2
// Readings: a community with H(X_k) = 0 (all n nodes) contributes 0; the
// admission test is false when {n11, n00} and {n01, n10} are the same
// multiset of counts (the two sides are then equal).
// Parity partially unpinned: the paper cites this measure without printing
// it; the tests pin identity, symmetry, relabelling, the zero cases and one
// worked example in closed form, not a value the paper gives.
// ---------------------------------------------------------------------------

static double hlog(i64 c, i64 n) {
    if (c <= 0) return 0.0;
    double p = (double)c / (double)n;
    return -p * std::log2(p);
}

static i64 intersect_sorted(const i32 *a, i64 na, const i32 *b, i64 nb) {
    i64 i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) i++;
        else if (a[i] > b[j]) j++;
        else { c++; i++; j++; }
    }
    return c;
}

static double cond_entropy_norm(i64 n, i64 cx, const i64 *xp, const i32 *xn, i64 cy, const i64 *yp,
                                const i32 *yn) {
    double total = 0.0;
    for (i64 k = 0; k < cx; k++) {
        i64 sx = xp[k + 1] - xp[k];
        double Hx = hlog(sx, n) + hlog(n - sx, n);
        double best = Hx;
        for (i64 l = 0; l < cy; l++) {
            i64 sy = yp[l + 1] - yp[l];
            i64 n11 = intersect_sorted(xn + xp[k], sx, yn + yp[l], sy);
            i64 n10 = sx - n11, n01 = sy - n11, n00 = n - n11 - n10 - n01;
            i64 lo1 = std::min(n11, n00), hi1 = std::max(n11, n00);
            i64 lo2 = std::min(n01, n10), hi2 = std::max(n01, n10);
            if (lo1 == lo2 && hi1 == hi2) continue;
            if (!(hlog(n11, n) + hlog(n00, n) > hlog(n01, n) + hlog(n10, n))) continue;
            double Hxy = hlog(n11, n) + hlog(n10, n) + hlog(n01, n) + hlog(n00, n);
            double Hy = hlog(sy, n) + hlog(n - sy, n);
            best = std::min(best, Hxy - Hy);
        }
        total += (Hx > 0.0) ? best / Hx : 0.0;
    }
    return total / (double)cx;
}

extern "C" double orc_nmi(i64 n, i64 cx, const i64 *xp, const i32 *xn, i64 cy, const i64 *yp, const i32 *yn) {
    if (cx <= 0 || cy <= 0 || n <= 0) return NAN;
    double hxy = cond_entropy_norm(n, cx, xp, xn, cy, yp, yn);
    double hyx = cond_entropy_norm(n, cy, yp, yn, cx, xp, xn);
    return 1.0 - 0.5 * (hxy + hyx);
}

// The same definition for covers too large for the pairwise list
// intersections above (tens of thousands of communities of hundreds of
// nodes).  Only the intersection sizes are obtained differently: n11 of
// (X_k, Y_l) is counted over the members of X_k and, for each, the Y
// communities holding it (a node -> communities index of Y); every other
// pair has n11 = 0.  Each pair is then evaluated by the same formulas, h()
// read from a table of hlog(c, n) for c = 0..n (the same values), the
// minimum over l is taken, and the per-k terms are summed in k order, so the
// result is the one cond_entropy_norm gives.  Threads split the k range.
static double cond_entropy_norm_indexed(i64 n, i64 cx, const i64 *xp, const i32 *xn, i64 cy, const i64 *yp,
                                        const i32 *yn, int n_threads) {
    std::vector<double> T(n + 1);
    for (i64 c = 0; c <= n; c++) T[c] = hlog(c, n);
    // node -> Y communities
    std::vector<i64> np(n + 1, 0);
    for (i64 l = 0; l < cy; l++)
        for (i64 j = yp[l]; j < yp[l + 1]; j++) np[yn[j] + 1]++;
    for (i64 v = 0; v < n; v++) np[v + 1] += np[v];
    std::vector<i64> nl(np[n]);
    {
        std::vector<i64> fill(np.begin(), np.end() - 1);
        for (i64 l = 0; l < cy; l++)
            for (i64 j = yp[l]; j < yp[l + 1]; j++) nl[fill[yn[j]]++] = l;
    }
    std::vector<double> term(cx);
    auto work = [&](i64 k0, i64 k1) {
        std::vector<i64> cnt(cy, 0);
        std::vector<i64> touched;
        for (i64 k = k0; k < k1; k++) {
            const i64 sx = xp[k + 1] - xp[k];
            const double Hx = T[sx] + T[n - sx];
            double best = Hx;
            touched.clear();
            for (i64 j = xp[k]; j < xp[k + 1]; j++) {
                const i32 v = xn[j];
                for (i64 q = np[v]; q < np[v + 1]; q++) {
                    if (cnt[nl[q]]++ == 0) touched.push_back(nl[q]);
                }
            }
            for (i64 l = 0; l < cy; l++) {
                const i64 sy = yp[l + 1] - yp[l];
                const i64 n11 = cnt[l];
                const i64 n10 = sx - n11, n01 = sy - n11, n00 = n - n11 - n10 - n01;
                const i64 lo1 = std::min(n11, n00), hi1 = std::max(n11, n00);
                const i64 lo2 = std::min(n01, n10), hi2 = std::max(n01, n10);
                if (lo1 == lo2 && hi1 == hi2) continue;
                if (!(T[n11] + T[n00] > T[n01] + T[n10])) continue;
                const double Hxy = T[n11] + T[n10] + T[n01] + T[n00];
                const double Hy = T[sy] + T[n - sy];
                best = std::min(best, Hxy - Hy);
            }
            for (i64 l : touched) cnt[l] = 0;
            term[k] = (Hx > 0.0) ? best / Hx : 0.0;
        }
    };
    const int t = std::max(1, n_threads);
    std::vector<std::thread> th;
    for (int i = 0; i < t; i++) th.emplace_back(work, cx * i / t, cx * (i + 1) / t);
    for (auto &x : th) x.join();
    double total = 0.0;
    for (i64 k = 0; k < cx; k++) total += term[k];
    return total / (double)cx;
}

extern "C" double orc_nmi_indexed(i64 n, i64 cx, const i64 *xp, const i32 *xn, i64 cy, const i64 *yp,
                                  const i32 *yn, int n_threads) {
    if (cx <= 0 || cy <= 0 || n <= 0) return NAN;
    double hxy = cond_entropy_norm_indexed(n, cx, xp, xn, cy, yp, yn, n_threads);
    double hyx = cond_entropy_norm_indexed(n, cy, yp, yn, cx, xp, xn, n_threads);
    return 1.0 - 0.5 * (hxy + hyx);
}

// Mean of the successive-scale NMI values inside a window of p scales centred
// on each scale i (scales i - (p-1)/2 ... i + p-1 - (p-1)/2, clipped to the
// list).  nmi has S-1 entries (nmi[j] compares scales j and j+1).
extern "C" int orc_window_means(const double *nmi, i32 S, i32 p, double *out) {
    if (S < 1 || p < 2) return ORC_EINVAL;
    for (i32 i = 0; i < S; i++) {
        i32 lo = i - (p - 1) / 2, hi = lo + p - 1;
        lo = std::max(lo, 0);
        hi = std::min(hi, S - 1);
        double s = 0.0;
        i32 c = 0;
        for (i32 j = lo; j + 1 <= hi; j++) { s += nmi[j]; c++; }
        out[i] = c ? s / c : NAN;
    }
    return ORC_OK;
}

// Scale list of Sec. 4 read as V_min + (A - V_min)(1 - log k / log X),
// k = 1..X: A first (finest), V_min last (coarsest).  X = 1 gives {A}.
extern "C" int orc_scales_logspaced(double vmin, double a, i32 x, double *out) {
    if (x < 1 || !(vmin > 0.0) || !(a >= vmin)) return ORC_EINVAL;
    if (x == 1) { out[0] = a; return ORC_OK; }
    double lx = std::log((double)x);
    for (i32 k = 1; k <= x; k++) out[k - 1] = vmin + (a - vmin) * (1.0 - std::log((double)k) / lx);
    return ORC_OK;
}

// ---------------------------------------------------------------------------
// The full method of Alg. 2 (with the modified growth of Alg. 3), written out
// sequentially in a fixed order:
//   * seeds (no initial communities given): candidates are the nodes with at
//     least two neighbours, taken in increasing `prio` (the random order of
//     the paper, passed in); a candidate still available becomes a seed and
//     makes its neighbours (rule 1) and also their neighbours (rule 2)
//     unavailable.  Community i starts as {seed_i}.  Given initial
//     communities, each is taken as it is, its first listed node as its seed.
//   * for every scale, while changes can be made:
//       - membership sets of the current communities;
//       - each community, in index order, against those sets: if it shares
//         at least eta * min(|c|, |c'|) nodes with another community c' it
//         is put on the check list unchanged (Alg. 3 pre-test); otherwise it
//         is grown once by Alg. 1 (grow pass, then prune passes if it added)
//         from its current members, its seed kept, and put on the check list
//         if its member set changed;
//       - membership sets again; every community on the check list, in index
//         order, counts shared nodes over its members in ascending id and,
//         for each member, over that node's communities in ascending index;
//         the first other community whose count reaches the threshold forms
//         a pair (c, c') to merge;
//       - merge rounds: the pairs are taken in list order into a round when
//         neither community is in the round yet; each taken pair merges c'
//         into c (union, c keeps its seed); in the remaining pairs c' is
//         renamed c and pairs that became (c, c) are dropped; repeat;
//       - a change is a grown community whose set changed or a merge.
//   * the communities left at the end of a scale (index order) are its
//     result and the start of the next scale.
// Merge criterion (Sec. 3): max(|A n B| / |A|, |A n B| / |B|) >= eta.
// ---------------------------------------------------------------------------

struct orc_full_result {
    std::vector<std::vector<std::vector<i32>>> comms;  // [scale][community] sorted members
    std::vector<std::vector<i32>> seeds;               // [scale][community]
    std::vector<std::vector<double>> f;                // [scale][community]
    std::vector<i64> iterations, merges, grown;        // [scale]
    std::vector<i32> initial_seeds;
};

static bool reaches(i64 count, i64 a, i64 b, double eta) { return (double)count >= eta * (double)std::min(a, b); }

// First community (other than c) whose shared-node count with c reaches the
// threshold in the scan order described above; -1 if none.
static i64 first_reaching(const std::vector<std::vector<i32>> &C, const std::vector<char> &alive,
                          const std::vector<std::vector<i64>> &memsets, i64 c, double eta) {
    std::unordered_map<i64, i64> count;
    for (i32 n : C[c])
        for (i64 o : memsets[n]) {
            if (o == c || !alive[o]) continue;
            i64 &k = ++count[o];
            if (reaches(k, (i64)C[c].size(), (i64)C[o].size(), eta)) return o;
        }
    return -1;
}

extern "C" int orc_full(const orc_graph *g, const double *alphas, i32 n_scales, int seed_rule, const i32 *prio,
                        const i64 *init_ptr, const i32 *init_nodes, i64 n_init, double eta, i64 max_iters,
                        orc_full_result **out) {
    *out = nullptr;
    if (n_scales < 1 || !(eta > 0.0) || eta > 1.0) return ORC_EINVAL;
    for (i32 s = 0; s < n_scales; s++)
        if (!(alphas[s] > 0.0) || !std::isfinite(alphas[s])) return ORC_EINVAL;
    const i64 n = g->n;
    std::vector<std::vector<i32>> C;
    std::vector<i32> seed;
    if (init_ptr) {
        for (i64 i = 0; i < n_init; i++) {
            std::vector<i32> m(init_nodes + init_ptr[i], init_nodes + init_ptr[i + 1]);
            if (m.empty()) return ORC_EINVAL;
            for (i32 v : m)
                if (v < 0 || v >= n) return ORC_EINVAL;
            seed.push_back(m[0]);
            std::sort(m.begin(), m.end());
            m.erase(std::unique(m.begin(), m.end()), m.end());
            C.push_back(m);
        }
    } else {
        if (seed_rule != 1 && seed_rule != 2) return ORC_EINVAL;
        std::vector<i32> order(n);
        for (i64 u = 0; u < n; u++) order[u] = (i32)u;
        std::sort(order.begin(), order.end(), [&](i32 a, i32 b) { return prio[a] < prio[b] || (prio[a] == prio[b] && a < b); });
        std::vector<char> avail(n, 0);
        for (i64 u = 0; u < n; u++) avail[u] = (g->rp[u + 1] - g->rp[u]) >= 2;
        for (i32 u : order) {
            if (!avail[u]) continue;
            seed.push_back(u);
            C.push_back({u});
            avail[u] = 0;
            for (i64 e = g->rp[u]; e < g->rp[u + 1]; e++) {
                const i32 v = g->col[e];
                avail[v] = 0;
                if (seed_rule == 2)
                    for (i64 f = g->rp[v]; f < g->rp[v + 1]; f++) avail[g->col[f]] = 0;
            }
        }
    }
    orc_full_result *r = new orc_full_result();
    r->initial_seeds = seed;
    int status = ORC_OK;
    for (i32 sc = 0; sc < n_scales; sc++) {
        const double alpha = alphas[sc];
        std::vector<char> alive(C.size(), 1);
        i64 it = 0, merges = 0, grown = 0;
        for (;; it++) {
            if (it >= max_iters) { status = ORC_ETIMEOUT; break; }
            auto build = [&](std::vector<std::vector<i64>> &ms) {
                ms.assign(n, {});
                for (i64 c = 0; c < (i64)C.size(); c++)
                    if (alive[c])
                        for (i32 v : C[c]) ms[v].push_back(c);
            };
            std::vector<std::vector<i64>> memsets;
            build(memsets);
            std::vector<char> check(C.size(), 0);
            bool changes = false;
            std::vector<std::vector<i32>> next = C;
            for (i64 c = 0; c < (i64)C.size(); c++) {
                if (!alive[c]) continue;
                if (first_reaching(C, alive, memsets, c, eta) >= 0) {
                    check[c] = 1;
                    continue;
                }
                UnitResult R;
                grow_unit(*g, seed[c], alpha, 1000000, R, C[c].data(), (i64)C[c].size(), true);
                if (R.status == ORC_EUNDECIDED) status = ORC_EUNDECIDED;
                grown++;
                if (R.members != C[c]) {
                    next[c] = R.members;
                    check[c] = 1;
                    changes = true;
                }
            }
            C.swap(next);
            build(memsets);
            std::vector<std::pair<i64, i64>> pairs;
            for (i64 c = 0; c < (i64)C.size(); c++)
                if (alive[c] && check[c]) {
                    const i64 o = first_reaching(C, alive, memsets, c, eta);
                    if (o >= 0) pairs.push_back({c, o});
                }
            while (!pairs.empty()) {
                std::vector<char> used(C.size(), 0);
                std::vector<std::pair<i64, i64>> round, rest;
                for (auto &pq : pairs) {
                    if (pq.first != pq.second && !used[pq.first] && !used[pq.second]) {
                        used[pq.first] = used[pq.second] = 1;
                        round.push_back(pq);
                    } else {
                        rest.push_back(pq);
                    }
                }
                std::vector<i64> into(C.size());
                for (i64 c = 0; c < (i64)C.size(); c++) into[c] = c;
                for (auto &pq : round) {
                    std::vector<i32> u;
                    std::set_union(C[pq.first].begin(), C[pq.first].end(), C[pq.second].begin(), C[pq.second].end(),
                                   std::back_inserter(u));
                    C[pq.first].swap(u);
                    C[pq.second].clear();
                    alive[pq.second] = 0;
                    into[pq.second] = pq.first;
                    merges++;
                    changes = true;
                }
                pairs.clear();
                for (auto &pq : rest) {
                    const i64 a = into[pq.first], b = into[pq.second];
                    if (a != b) pairs.push_back({a, b});
                }
            }
            if (!changes) break;
        }
        // compact: the communities left, in index order
        std::vector<std::vector<i32>> keep;
        std::vector<i32> kseed;
        for (i64 c = 0; c < (i64)C.size(); c++)
            if (alive[c]) {
                keep.push_back(C[c]);
                kseed.push_back(seed[c]);
            }
        C.swap(keep);
        seed.swap(kseed);
        std::vector<double> fs;
        for (auto &m : C) {
            i64 K = 0, V = 0;
            std::unordered_map<i32, char> in;
            for (i32 v : m) in[v] = 1;
            for (i32 v : m) {
                V += g->k[v];
                for (i64 e = g->rp[v]; e < g->rp[v + 1]; e++)
                    if (in.count(g->col[e])) K += g->wt(e);
            }
            fs.push_back(fitness(K, V, alpha, g->unit_exp));
        }
        r->comms.push_back(C);
        r->seeds.push_back(seed);
        r->f.push_back(fs);
        r->iterations.push_back(it);
        r->merges.push_back(merges);
        r->grown.push_back(grown);
        if (status == ORC_ETIMEOUT) break;
    }
    *out = r;
    return status;
}

extern "C" void orc_full_destroy(orc_full_result *r) { delete r; }

// Sizes of scale s: communities, member entries.
extern "C" int orc_full_sizes(const orc_full_result *r, i32 s, i64 *n_comms, i64 *n_nodes, i64 *iters, i64 *merges) {
    if (s < 0 || s >= (i32)r->comms.size()) return ORC_EINVAL;
    *n_comms = (i64)r->comms[s].size();
    i64 t = 0;
    for (auto &m : r->comms[s]) t += (i64)m.size();
    *n_nodes = t;
    if (iters) *iters = r->iterations[s];
    if (merges) *merges = r->merges[s];
    return ORC_OK;
}

extern "C" int orc_full_get(const orc_full_result *r, i32 s, i64 *ptr, i32 *nodes, i32 *seeds, double *f) {
    if (s < 0 || s >= (i32)r->comms.size()) return ORC_EINVAL;
    ptr[0] = 0;
    for (size_t c = 0; c < r->comms[s].size(); c++) {
        const auto &m = r->comms[s][c];
        std::copy(m.begin(), m.end(), nodes + ptr[c]);
        ptr[c + 1] = ptr[c] + (i64)m.size();
        if (seeds) seeds[c] = r->seeds[s][c];
        if (f) f[c] = r->f[s][c];
    }
    return ORC_OK;
}

extern "C" i64 orc_full_n_seeds(const orc_full_result *r, i32 *seeds) {
    if (seeds) std::copy(r->initial_seeds.begin(), r->initial_seeds.end(), seeds);
    return (i64)r->initial_seeds.size();
}

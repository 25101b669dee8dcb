// paulib_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously-correct CPU definition of the Pauli-sum product and
// its canonical form.  It exists so the tests, the smoke check and the CPU
// baseline leg of the benchmark have something independent to compare the GPU
// library against.  Nothing in the product library links, includes or calls
// this file, and this file shares no code with the library.
//
// What it computes (PauLIB, Sec. III):
//   * Single-qubit products come from the paper's table of Pauli products
//     (Sec. III-A): I is neutral, P*P = I, and
//       XY = iZ, YZ = iX, ZX = iY,   YX = -iZ, ZY = -iX, XZ = -iY.
//   * A Pauli string product is taken qubit by qubit with that table and the
//     phases are accumulated into one global phase i^k (Sec. III-A, the worked
//     example (XIZ)(ZIX) = YIY).
//   * Qubit letters are decoded from the binary symplectic (x|z) bits of
//     Table I: I=(0,0), Z=(0,1), X=(1,0), Y=(1,1).  Qubit q lives in word q/64
//     (Sec. III-G), bit q%64 (least significant bit = lowest qubit; the paper
//     fixes only the word index, this bit order is our reading).
//   * A Pauli sum is sum_j c_j P_j with complex c_j (Eq. 2).
//   * The product of two sums is the outer product: every left term times
//     every right term (Sec. IV-B/IV-C).  Raw order: the block of right term j
//     holds the products of all left terms i, i.e. raw index j*|A| + i.
//   * Canonical form = sort by a lexicographic key of the packed words and
//     merge adjacent duplicates by adding coefficients (Sec. III-H).  The key
//     is (x_0..x_{W-1}, z_0..z_{W-1}) compared as unsigned 64-bit words, word
//     0 most significant (our reading: the paper names a lexicographic key over
//     the packed words without fixing the word order).  Terms whose merged
//     coefficient is zero are kept (the paper drops terms only in truncation).
//
// Arithmetic: FP64 throughout, built with -ffp-contract=off.  Duplicate
// coefficients are summed with Neumaier's compensated summation so the oracle's
// own rounding error stays far below the tolerance the GPU path is held to.
// Every merged key also reports sum |c_a||c_b| over its contributions and the
// contribution count, which the tolerance and the tests use.
//
// Data layout at this interface: struct of arrays as in the paper's PauliSumSoA
// (Sec. IV-A): word w of term t at x[w*n_terms + t]; complex coefficients are
// interleaved (re, im); optional per-term phase exponents k in {0,1,2,3} mean
// the term is i^k * c * P.
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <algorithm>
#include <map>
#include <thread>
#include <vector>

namespace {

enum Letter { I_ = 0, X_ = 1, Y_ = 2, Z_ = 3 };

struct Prod { int letter; int k; };

// The paper's single-qubit multiplication table (Sec. III-A), written out
// entry by entry.  k is the exponent of i in the phase.
Prod letter_product(int a, int b) {
    if (a == I_) return {b, 0};
    if (b == I_) return {a, 0};
    if (a == b) return {I_, 0};
    if (a == X_ && b == Y_) return {Z_, 1};   // XY =  iZ
    if (a == Y_ && b == Z_) return {X_, 1};   // YZ =  iX
    if (a == Z_ && b == X_) return {Y_, 1};   // ZX =  iY
    if (a == Y_ && b == X_) return {Z_, 3};   // YX = -iZ
    if (a == Z_ && b == Y_) return {X_, 3};   // ZY = -iX
    if (a == X_ && b == Z_) return {Y_, 3};   // XZ = -iY
    std::abort();
}

// Table I: (x-bit, z-bit) -> letter.
int decode(int xbit, int zbit) {
    if (!xbit && !zbit) return I_;
    if (!xbit && zbit) return Z_;
    if (xbit && !zbit) return X_;
    return Y_;
}
void encode(int letter, int* xbit, int* zbit) {
    *xbit = (letter == X_ || letter == Y_) ? 1 : 0;
    *zbit = (letter == Z_ || letter == Y_) ? 1 : 0;
}

int words_for(int n) { return (n + 63) / 64; }

int get_bit(const uint64_t* w, int q) { return (int)((w[q / 64] >> (q % 64)) & 1ull); }
void set_bit(uint64_t* w, int q) { w[q / 64] |= (1ull << (q % 64)); }

// One Pauli string held as per-word arrays of length W.
struct Str { std::vector<uint64_t> x, z; };

Str load_term(int W, int64_t n_terms, const uint64_t* xs, const uint64_t* zs, int64_t t) {
    Str s; s.x.assign(W, 0); s.z.assign(W, 0);
    for (int w = 0; w < W; ++w) { s.x[w] = xs[(int64_t)w * n_terms + t]; s.z[w] = zs[(int64_t)w * n_terms + t]; }
    return s;
}

// Product of two strings, qubit by qubit (Sec. III-A): returns k with
// P_a P_b = i^k P_out.
int string_product(int n, const Str& a, const Str& b, Str* out) {
    int W = words_for(n);
    out->x.assign(W, 0); out->z.assign(W, 0);
    int k = 0;
    for (int q = 0; q < n; ++q) {
        int la = decode(get_bit(a.x.data(), q), get_bit(a.z.data(), q));
        int lb = decode(get_bit(b.x.data(), q), get_bit(b.z.data(), q));
        Prod p = letter_product(la, lb);
        k = (k + p.k) % 4;
        int xb, zb; encode(p.letter, &xb, &zb);
        if (xb) set_bit(out->x.data(), q);
        if (zb) set_bit(out->z.data(), q);
    }
    return k;
}

// Key = (x_0..x_{W-1}, z_0..z_{W-1}); std::vector's operator< is the
// lexicographic comparison with unsigned 64-bit elements.
std::vector<uint64_t> key_of(const Str& s) {
    std::vector<uint64_t> k(s.x);
    k.insert(k.end(), s.z.begin(), s.z.end());
    return k;
}

struct Cplx { double re, im; };

Cplx cmul(Cplx a, Cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// Multiply by i^k exactly (a swap and/or sign flips, no rounding).
Cplx rot(Cplx c, int k) {
    switch (k & 3) {
        case 0: return c;
        case 1: return {-c.im, c.re};
        case 2: return {-c.re, -c.im};
        default: return {c.im, -c.re};
    }
}

// Neumaier's compensated sum (improved Kahan-Babuska).
struct Neumaier {
    double s = 0.0, c = 0.0;
    void add(double v) {
        double t = s + v;
        if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v; else c += (v - t) + s;
        s = t;
    }
    double value() const { return s + c; }
};

struct Acc { Neumaier re, im; double abs_sum = 0.0; int64_t count = 0; };

struct Result {
    int n = 0, W = 0;
    std::vector<std::vector<uint64_t>> keys;
    std::vector<double> coef;      // interleaved re, im
    std::vector<double> abs_sum;
    std::vector<int64_t> count;
};

void emit(const std::map<std::vector<uint64_t>, Acc>& m, Result* r) {
    for (const auto& kv : m) {
        r->keys.push_back(kv.first);
        r->coef.push_back(kv.second.re.value());
        r->coef.push_back(kv.second.im.value());
        r->abs_sum.push_back(kv.second.abs_sum);
        r->count.push_back(kv.second.count);
    }
}

Cplx load_coef(const double* c, int64_t t) { return {c[2 * t], c[2 * t + 1]}; }

}  // namespace

extern "C" {

int oracle_abi_version(void) { return 2; }

// Single-qubit product; letters 0=I, 1=X, 2=Y, 3=Z.
void oracle_letter_product(int a, int b, int* out_letter, int* out_k) {
    Prod p = letter_product(a, b);
    *out_letter = p.letter; *out_k = p.k;
}

// Product of two single strings given as W-word arrays; writes the product
// string and returns k (P_a P_b = i^k P_out).
int oracle_string_product(int n, const uint64_t* xa, const uint64_t* za, const uint64_t* xb,
                          const uint64_t* zb, uint64_t* xo, uint64_t* zo) {
    int W = words_for(n);
    Str a, b, o;
    a.x.assign(xa, xa + W); a.z.assign(za, za + W);
    b.x.assign(xb, xb + W); b.z.assign(zb, zb + W);
    int k = string_product(n, a, b, &o);
    for (int w = 0; w < W; ++w) { xo[w] = o.x[w]; zo[w] = o.z[w]; }
    return k;
}

// Raw outer product (Sec. IV-C): output slot j*na + i holds a_i * b_j with
// key a_i XOR b_j, phase k = k_a + k_b + k_pair (mod 4) and the unrotated
// coefficient c_a * c_b.  ka/kb may be NULL (all zero).  Output is SoA with
// n_out = na*nb terms.
void oracle_multiply_raw(int n, int64_t na, const uint64_t* ax, const uint64_t* az, const double* ac,
                         const uint8_t* ka, int64_t nb, const uint64_t* bx, const uint64_t* bz,
                         const double* bc, const uint8_t* kb, uint64_t* ox, uint64_t* oz, double* oc,
                         uint8_t* ok) {
    int W = words_for(n);
    int64_t nout = na * nb;
    for (int64_t j = 0; j < nb; ++j) {
        Str b = load_term(W, nb, bx, bz, j);
        for (int64_t i = 0; i < na; ++i) {
            Str a = load_term(W, na, ax, az, i);
            Str o;
            int k = string_product(n, a, b, &o);
            k = (k + (ka ? ka[i] : 0) + (kb ? kb[j] : 0)) % 4;
            int64_t t = j * na + i;
            for (int w = 0; w < W; ++w) { ox[(int64_t)w * nout + t] = o.x[w]; oz[(int64_t)w * nout + t] = o.z[w]; }
            Cplx c = cmul(load_coef(ac, i), load_coef(bc, j));
            oc[2 * t] = c.re; oc[2 * t + 1] = c.im;
            ok[t] = (uint8_t)k;
        }
    }
}

// Canonical product: C = sum_i sum_j c_a_i c_b_j (P_a_i P_b_j), one term per
// distinct product string, in ascending key order.  Returns an opaque handle.
void* oracle_multiply_canonical(int n, int64_t na, const uint64_t* ax, const uint64_t* az,
                                const double* ac, const uint8_t* ka, int64_t nb, const uint64_t* bx,
                                const uint64_t* bz, const double* bc, const uint8_t* kb) {
    int W = words_for(n);
    std::map<std::vector<uint64_t>, Acc> m;
    for (int64_t j = 0; j < nb; ++j) {
        Str b = load_term(W, nb, bx, bz, j);
        Cplx cb = load_coef(bc, j);
        for (int64_t i = 0; i < na; ++i) {
            Str a = load_term(W, na, ax, az, i);
            Str o;
            int k = string_product(n, a, b, &o);
            k = (k + (ka ? ka[i] : 0) + (kb ? kb[j] : 0)) % 4;
            Cplx ca = load_coef(ac, i);
            Cplx c = rot(cmul(ca, cb), k);
            Acc& acc = m[key_of(o)];
            acc.re.add(c.re); acc.im.add(c.im);
            acc.abs_sum += std::hypot(ca.re, ca.im) * std::hypot(cb.re, cb.im);
            acc.count += 1;
        }
    }
    Result* r = new Result; r->n = n; r->W = W;
    emit(m, r);
    return r;
}

// Canonical form of one sum (sort by key, merge duplicates); a term with phase
// k contributes i^k c.  kin may be NULL.
void* oracle_compress(int n, int64_t nt, const uint64_t* xs, const uint64_t* zs, const double* cs,
                      const uint8_t* kin) {
    int W = words_for(n);
    std::map<std::vector<uint64_t>, Acc> m;
    for (int64_t t = 0; t < nt; ++t) {
        Str s = load_term(W, nt, xs, zs, t);
        Cplx c0 = load_coef(cs, t);
        Cplx c = rot(c0, kin ? kin[t] : 0);
        Acc& acc = m[key_of(s)];
        acc.re.add(c.re); acc.im.add(c.im);
        acc.abs_sum += std::hypot(c0.re, c0.im);
        acc.count += 1;
    }
    Result* r = new Result; r->n = n; r->W = W;
    emit(m, r);
    return r;
}

// Canonical product restricted to the key range [lo, hi) (lo or hi NULL:
// open at that end), with the right-hand terms split into nthreads contiguous
// blocks, one std::thread each.  Used to check full-size products one key range
// at a time, so host memory stays bounded: the results of consecutive ranges,
// concatenated, are the canonical sum.
//
// A pair is selected by the word-wise XOR of its factors' keys (the key of a
// product string; tests/test_oracle_pins.py pins the key set {a_i XOR b_j}
// against Kronecker matrices).  Each selected pair is then multiplied qubit by
// qubit from the letter table exactly as in oracle_multiply_canonical, and its
// letter-table key must equal the XOR (else the call aborts).  Sort and
// combine (Sec. III-H) is done literally: every thread lists its selected
// products (key, pair, coefficient), sorts the list by (key, j, i), and the
// sorted lists are merged in key order; equal keys are summed with Neumaier's
// compensated sum in (j, i) order, so the result does not depend on thread
// timing.
namespace {
struct RangeRec { int64_t j, i; double re, im, abs; };
struct RangeList {
    int W2 = 0;
    std::vector<uint64_t> keys;   // W2 words per record
    std::vector<RangeRec> recs;
    std::vector<int64_t> order;   // records sorted by (key, j, i)
    bool less(int64_t p, int64_t q) const {
        const uint64_t* a = &keys[(size_t)p * W2];
        const uint64_t* b = &keys[(size_t)q * W2];
        for (int w = 0; w < W2; ++w)
            if (a[w] != b[w]) return a[w] < b[w];
        if (recs[p].j != recs[q].j) return recs[p].j < recs[q].j;
        return recs[p].i < recs[q].i;
    }
};
}  // namespace

void* oracle_multiply_canonical_range(int n, int64_t na, const uint64_t* ax, const uint64_t* az,
                                      const double* ac, const uint8_t* ka, int64_t nb, const uint64_t* bx,
                                      const uint64_t* bz, const double* bc, const uint8_t* kb,
                                      const uint64_t* lo, const uint64_t* hi, int nthreads) {
    const int W = words_for(n);
    if (nthreads < 1) nthreads = 1;
    std::vector<uint64_t> klo, khi;
    if (lo) klo.assign(lo, lo + 2 * W);
    if (hi) khi.assign(hi, hi + 2 * W);
    std::vector<Str> as;
    as.reserve(na);
    for (int64_t i = 0; i < na; ++i) as.push_back(load_term(W, na, ax, az, i));
    std::vector<RangeList> lists(nthreads);
    auto work = [&](int t) {
        const int64_t j0 = nb * t / nthreads, j1 = nb * (t + 1) / nthreads;
        RangeList& L = lists[t];
        L.W2 = 2 * W;
        std::vector<uint64_t> kx(2 * W);
        Str o;
        for (int64_t j = j0; j < j1; ++j) {
            Str b = load_term(W, nb, bx, bz, j);
            Cplx cb = load_coef(bc, j);
            for (int64_t i = 0; i < na; ++i) {
                for (int w = 0; w < W; ++w) {
                    kx[w] = as[i].x[w] ^ b.x[w];
                    kx[W + w] = as[i].z[w] ^ b.z[w];
                }
                if (lo && kx < klo) continue;
                if (hi && !(kx < khi)) continue;
                int k = string_product(n, as[i], b, &o);
                for (int w = 0; w < W; ++w)
                    if (o.x[w] != kx[w] || o.z[w] != kx[W + w]) std::abort();
                k = (k + (ka ? ka[i] : 0) + (kb ? kb[j] : 0)) % 4;
                Cplx ca = load_coef(ac, i);
                Cplx c = rot(cmul(ca, cb), k);
                L.keys.insert(L.keys.end(), kx.begin(), kx.end());
                L.recs.push_back(RangeRec{j, i, c.re, c.im, std::hypot(ca.re, ca.im) * std::hypot(cb.re, cb.im)});
            }
        }
        L.order.resize(L.recs.size());
        for (size_t q = 0; q < L.order.size(); ++q) L.order[q] = (int64_t)q;
        std::sort(L.order.begin(), L.order.end(), [&L](int64_t p, int64_t q) { return L.less(p, q); });
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
    // merge the sorted lists in key order (threads hold disjoint j blocks in
    // increasing order, so among equal keys the lower thread comes first)
    Result* r = new Result; r->n = n; r->W = W;
    std::vector<size_t> cur(nthreads, 0);
    const uint64_t* last = nullptr;
    Acc acc;
    auto flush = [&]() {
        if (!last) return;
        r->keys.emplace_back(last, last + 2 * W);
        r->coef.push_back(acc.re.value());
        r->coef.push_back(acc.im.value());
        r->abs_sum.push_back(acc.abs_sum);
        r->count.push_back(acc.count);
        acc = Acc();
    };
    for (;;) {
        int best = -1;
        const uint64_t* bk = nullptr;
        for (int t = 0; t < nthreads; ++t) {
            if (cur[t] >= lists[t].order.size()) continue;
            const uint64_t* k = &lists[t].keys[(size_t)lists[t].order[cur[t]] * 2 * W];
            if (best < 0 || std::lexicographical_compare(k, k + 2 * W, bk, bk + 2 * W)) {
                best = t;
                bk = k;
            }
        }
        if (best < 0) break;
        const RangeRec& rec = lists[best].recs[(size_t)lists[best].order[cur[best]]];
        if (!last || !std::equal(bk, bk + 2 * W, last)) {
            flush();
            last = bk;
        }
        acc.re.add(rec.re);
        acc.im.add(rec.im);
        acc.abs_sum += rec.abs;
        acc.count += 1;
        ++cur[best];
    }
    flush();
    return r;
}

int64_t oracle_result_size(const void* h) { return (int64_t)static_cast<const Result*>(h)->keys.size(); }

// Copies a result out as SoA words, interleaved coefficients, per-term
// sum |contribution| and contribution counts (any output pointer may be NULL).
void oracle_result_copy(const void* h, uint64_t* ox, uint64_t* oz, double* oc, double* oabs,
                        int64_t* ocount) {
    const Result* r = static_cast<const Result*>(h);
    int64_t u = (int64_t)r->keys.size();
    for (int64_t t = 0; t < u; ++t) {
        for (int w = 0; w < r->W; ++w) {
            if (ox) ox[(int64_t)w * u + t] = r->keys[t][w];
            if (oz) oz[(int64_t)w * u + t] = r->keys[t][r->W + w];
        }
        if (oc) { oc[2 * t] = r->coef[2 * t]; oc[2 * t + 1] = r->coef[2 * t + 1]; }
        if (oabs) oabs[t] = r->abs_sum[t];
        if (ocount) ocount[t] = r->count[t];
    }
}

void oracle_result_free(void* h) { delete static_cast<Result*>(h); }

// Coefficient of given product strings in A*B, one query at a time, straight
// from the definition: every pair (i, j) with a_i XOR b_j equal to the query
// contributes i^k c_a c_b.  For each query and each left term i the matching
// right terms are found by looking up (query XOR a_i) in an ordered map of B's
// keys.  Queries are SoA (nq terms).  Writes coefficient, sum |contribution|
// and contribution count per query.
void oracle_query_product_coeffs(int n, int64_t na, const uint64_t* ax, const uint64_t* az,
                                 const double* ac, const uint8_t* ka, int64_t nb, const uint64_t* bx,
                                 const uint64_t* bz, const double* bc, const uint8_t* kb, int64_t nq,
                                 const uint64_t* qx, const uint64_t* qz, double* oc, double* oabs,
                                 int64_t* ocount) {
    int W = words_for(n);
    std::map<std::vector<uint64_t>, std::vector<int64_t>> bmap;
    for (int64_t j = 0; j < nb; ++j) bmap[key_of(load_term(W, nb, bx, bz, j))].push_back(j);
    std::vector<Str> as;
    as.reserve(na);
    for (int64_t i = 0; i < na; ++i) as.push_back(load_term(W, na, ax, az, i));
    for (int64_t q = 0; q < nq; ++q) {
        Str want = load_term(W, nq, qx, qz, q);
        Acc acc;
        for (int64_t i = 0; i < na; ++i) {
            Str need; need.x.assign(W, 0); need.z.assign(W, 0);
            for (int w = 0; w < W; ++w) { need.x[w] = want.x[w] ^ as[i].x[w]; need.z[w] = want.z[w] ^ as[i].z[w]; }
            auto it = bmap.find(key_of(need));
            if (it == bmap.end()) continue;
            for (int64_t j : it->second) {
                Str b = load_term(W, nb, bx, bz, j);
                Str o;
                int k = string_product(n, as[i], b, &o);
                k = (k + (ka ? ka[i] : 0) + (kb ? kb[j] : 0)) % 4;
                Cplx ca = load_coef(ac, i), cb = load_coef(bc, j);
                Cplx c = rot(cmul(ca, cb), k);
                acc.re.add(c.re); acc.im.add(c.im);
                acc.abs_sum += std::hypot(ca.re, ca.im) * std::hypot(cb.re, cb.im);
                acc.count += 1;
            }
        }
        oc[2 * q] = acc.re.value(); oc[2 * q + 1] = acc.im.value();
        oabs[q] = acc.abs_sum; ocount[q] = acc.count;
    }
}

// Compensated sum of n doubles (exposed so the tests can pin the summation
// against a correctly rounded library sum).
// ---------------------------------------------------------------- gates
//
// Conjugation Q' = U Q U^dagger of every term by a Clifford gate (Sec. III-B,
// Eq. for the conjugation; gate application of Sec. V-B): the gate's 2x2 or 4x4
// matrix is applied to the local Pauli matrix of the qubits it acts on, and
// the image is decomposed back into Pauli letters by traces.  Gates: 0 = H,
// 1 = S, 2 = CNOT (control q1, target q2), 3 = CZ (q1, q2).  Terms keep their
// order; the output coefficient folds in the input phase i^k and the image's
// sign.  Matrices act with qubit q1 as the first tensor factor.

namespace {

struct CM { double re, im; };
CM cm(double r, double i) { return {r, i}; }
CM cadd(CM a, CM b) { return {a.re + b.re, a.im + b.im}; }
CM cmulm(CM a, CM b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
CM cconj(CM a) { return {a.re, -a.im}; }

// The paper's Pauli matrices (Sec. III-A): I, X, Y = [[0,-i],[i,0]], Z.
void pauli_matrix(int letter, CM m[2][2]) {
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) m[r][c] = cm(0, 0);
    switch (letter) {
        case I_: m[0][0] = cm(1, 0); m[1][1] = cm(1, 0); break;
        case X_: m[0][1] = cm(1, 0); m[1][0] = cm(1, 0); break;
        case Y_: m[0][1] = cm(0, -1); m[1][0] = cm(0, 1); break;
        default: m[0][0] = cm(1, 0); m[1][1] = cm(-1, 0); break;
    }
}

// d x d matrices, d = 2 or 4, stored row-major in a 16-entry array.
void local_matrix(const int* letters, int nq, CM* out) {
    CM a[2][2], b[2][2];
    pauli_matrix(letters[0], a);
    if (nq == 1) {
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) out[r * 2 + c] = a[r][c];
        return;
    }
    pauli_matrix(letters[1], b);
    for (int r1 = 0; r1 < 2; ++r1)
        for (int c1 = 0; c1 < 2; ++c1)
            for (int r2 = 0; r2 < 2; ++r2)
                for (int c2 = 0; c2 < 2; ++c2) out[(r1 * 2 + r2) * 4 + (c1 * 2 + c2)] = cmulm(a[r1][c1], b[r2][c2]);
}

void gate_matrix(int gate, CM* u) {
    const double h = 1.0 / std::sqrt(2.0);
    for (int q = 0; q < 16; ++q) u[q] = cm(0, 0);
    switch (gate) {
        case 0: u[0] = cm(h, 0); u[1] = cm(h, 0); u[2] = cm(h, 0); u[3] = cm(-h, 0); break;  // H
        case 1: u[0] = cm(1, 0); u[3] = cm(0, 1); break;                                      // S = diag(1, i)
        case 2:  // CNOT: |c t> -> |c, t xor c>
            u[0 * 4 + 0] = cm(1, 0); u[1 * 4 + 1] = cm(1, 0); u[3 * 4 + 2] = cm(1, 0); u[2 * 4 + 3] = cm(1, 0);
            break;
        default:  // CZ = diag(1, 1, 1, -1)
            u[0] = cm(1, 0); u[5] = cm(1, 0); u[10] = cm(1, 0); u[15] = cm(-1, 0);
            break;
    }
}

void matmul(const CM* a, const CM* b, CM* c, int d) {
    for (int r = 0; r < d; ++r)
        for (int k = 0; k < d; ++k) {
            CM s = cm(0, 0);
            for (int q = 0; q < d; ++q) s = cadd(s, cmulm(a[r * d + q], b[q * d + k]));
            c[r * d + k] = s;
        }
}

// Image of the local letters under the gate: new letters and the exponent e
// of the factor i^e (the image is i^e times a Pauli product).
void conjugate_local(int gate, const int* letters, int nq, int* out_letters, int* e) {
    const int d = nq == 1 ? 2 : 4;
    CM u[16], m[16], t[16], r[16], ud[16];
    gate_matrix(gate, u);
    local_matrix(letters, nq, m);
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) ud[a * d + b] = cconj(u[b * d + a]);
    matmul(u, m, t, d);
    matmul(t, ud, r, d);
    int found = 0;
    for (int cand = 0; cand < (nq == 1 ? 4 : 16); ++cand) {
        int cl[2] = {nq == 1 ? cand : cand / 4, cand % 4};
        CM p[16];
        local_matrix(cl, nq, p);
        CM tr = cm(0, 0);  // Tr(p^dagger r) / d
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) tr = cadd(tr, cmulm(cconj(p[b * d + a]), r[b * d + a]));
        tr.re /= d; tr.im /= d;
        if (std::hypot(tr.re, tr.im) < 0.5) continue;
        int k;
        if (tr.re > 0.5) k = 0; else if (tr.im > 0.5) k = 1; else if (tr.re < -0.5) k = 2; else k = 3;
        out_letters[0] = cl[0];
        if (nq == 2) out_letters[1] = cl[1];
        *e = k;
        ++found;
    }
    if (found != 1) std::abort();
}

}  // namespace

void oracle_apply_clifford(int n, int64_t nt, const uint64_t* xs, const uint64_t* zs, const double* cs,
                           const uint8_t* kin, int gate, int q1, int q2, uint64_t* ox, uint64_t* oz,
                           double* oc) {
    const int W = words_for(n);
    const int nq = gate >= 2 ? 2 : 1;
    for (int64_t t = 0; t < nt; ++t) {
        Str s = load_term(W, nt, xs, zs, t);
        int letters[2] = {decode(get_bit(s.x.data(), q1), get_bit(s.z.data(), q1)),
                          nq == 2 ? decode(get_bit(s.x.data(), q2), get_bit(s.z.data(), q2)) : 0};
        int nl[2] = {0, 0}, e = 0;
        conjugate_local(gate, letters, nq, nl, &e);
        const int qs[2] = {q1, q2};
        for (int j = 0; j < nq; ++j) {
            int xb, zb;
            encode(nl[j], &xb, &zb);
            const uint64_t bit = 1ull << (qs[j] % 64);
            s.x[qs[j] / 64] = xb ? (s.x[qs[j] / 64] | bit) : (s.x[qs[j] / 64] & ~bit);
            s.z[qs[j] / 64] = zb ? (s.z[qs[j] / 64] | bit) : (s.z[qs[j] / 64] & ~bit);
        }
        for (int w = 0; w < W; ++w) { ox[(int64_t)w * nt + t] = s.x[w]; oz[(int64_t)w * nt + t] = s.z[w]; }
        Cplx c = rot(load_coef(cs, t), (kin ? kin[t] : 0) + e);
        oc[2 * t] = c.re; oc[2 * t + 1] = c.im;
    }
}

// Conjugation by the Pauli rotation U_P(theta) = exp(-i theta P / 2) (Sec.
// III-B): a term Q that commutes with P is kept; one that anti-commutes
// becomes cos(theta) Q - i sin(theta) P Q (Eq. for the non-Clifford case).
// Whether Q and P commute is read qubit by qubit: they anti-commute at a qubit
// where both letters are non-identity and differ, and Q, P anti-commute when
// that happens at an odd number of qubits (Sec. III-F).  The result is merged
// into canonical form (Sec. III-H) and, when threshold > 0, merged terms with
// |c| < threshold are dropped (truncation, Sec. III-B).  P is one string
// (W words of x and of z).
void* oracle_rotate(int n, int64_t nt, const uint64_t* xs, const uint64_t* zs, const double* cs,
                    const uint8_t* kin, const uint64_t* px, const uint64_t* pz, double theta,
                    double threshold) {
    const int W = words_for(n);
    Str P;
    P.x.assign(px, px + W);
    P.z.assign(pz, pz + W);
    const double cth = std::cos(theta), sth = std::sin(theta);
    std::map<std::vector<uint64_t>, Acc> m;
    auto add = [&](const Str& s, Cplx c) {
        Acc& acc = m[key_of(s)];
        acc.re.add(c.re); acc.im.add(c.im);
        acc.abs_sum += std::hypot(c.re, c.im);
        acc.count += 1;
    };
    for (int64_t t = 0; t < nt; ++t) {
        Str q = load_term(W, nt, xs, zs, t);
        Cplx c = rot(load_coef(cs, t), kin ? kin[t] : 0);
        int anti = 0;
        for (int b = 0; b < n; ++b) {
            int lp = decode(get_bit(P.x.data(), b), get_bit(P.z.data(), b));
            int lq = decode(get_bit(q.x.data(), b), get_bit(q.z.data(), b));
            if (lp != I_ && lq != I_ && lp != lq) anti ^= 1;
        }
        if (!anti) { add(q, c); continue; }
        add(q, Cplx{cth * c.re, cth * c.im});
        Str pq;
        int k = string_product(n, P, q, &pq);           // P Q = i^k R
        Cplx s2 = rot(Cplx{sth * c.re, sth * c.im}, 3 + k);  // -i sin(theta) c i^k
        add(pq, s2);
    }
    Result* r = new Result; r->n = n; r->W = W;
    for (const auto& kv : m) {
        const double re = kv.second.re.value(), im = kv.second.im.value();
        if (threshold > 0 && std::hypot(re, im) < threshold) continue;
        r->keys.push_back(kv.first);
        r->coef.push_back(re);
        r->coef.push_back(im);
        r->abs_sum.push_back(kv.second.abs_sum);
        r->count.push_back(kv.second.count);
    }
    return r;
}

// Element-wise products a_t * b_t of two equally long lists of terms (the
// paper's single Pauli multiplication, Sec. III-A/III-E, applied pair by
// pair): output t is the product string with phase exponent k_t (including
// both inputs' phases) and coefficient c_a c_b.
void oracle_multiply_pairwise(int n, int64_t nt, const uint64_t* ax, const uint64_t* az, const double* ac,
                              const uint8_t* ka, const uint64_t* bx, const uint64_t* bz, const double* bc,
                              const uint8_t* kb, uint64_t* ox, uint64_t* oz, double* oc, uint8_t* ok) {
    const int W = words_for(n);
    for (int64_t t = 0; t < nt; ++t) {
        Str a = load_term(W, nt, ax, az, t), b = load_term(W, nt, bx, bz, t), o;
        const int k = string_product(n, a, b, &o);
        for (int w = 0; w < W; ++w) { ox[(int64_t)w * nt + t] = o.x[w]; oz[(int64_t)w * nt + t] = o.z[w]; }
        const Cplx c = cmul(load_coef(ac, t), load_coef(bc, t));
        oc[2 * t] = c.re; oc[2 * t + 1] = c.im;
        ok[t] = (uint8_t)((k + (ka ? ka[t] : 0) + (kb ? kb[t] : 0)) & 3);
    }
}

double oracle_compensated_sum(int64_t n, const double* v) {
    Neumaier s;
    for (int64_t t = 0; t < n; ++t) s.add(v[t]);
    return s.value();
}

// Greedy commutation grouping (Sec. V-D; the sequential variant of Sec.
// IV-C): the terms are visited in their order and each joins the first group
// (groups numbered in the order they were opened) all of whose members commute
// with it, or opens a new group when no group qualifies.  Two strings commute
// when the qubits at which their letters anti-commute (both non-identity and
// different) are even in number (Sec. III-A), read here letter by letter.
// group[t] receives the group of term t; the return value is the number of
// groups.  Coefficients and phases play no part.
int64_t oracle_group_commuting(int n, int64_t nt, const uint64_t* xs, const uint64_t* zs, int32_t* group) {
    const int W = words_for(n);
    std::vector<uint8_t> let((size_t)nt * n);
    for (int64_t t = 0; t < nt; ++t) {
        const Str s = load_term(W, nt, xs, zs, t);
        for (int b = 0; b < n; ++b)
            let[(size_t)t * n + b] = (uint8_t)decode(get_bit(s.x.data(), b), get_bit(s.z.data(), b));
    }
    auto commute = [&](int64_t a, int64_t b) {
        const uint8_t* la = &let[(size_t)a * n];
        const uint8_t* lb = &let[(size_t)b * n];
        int anti = 0;
        for (int q = 0; q < n; ++q)
            if (la[q] != I_ && lb[q] != I_ && la[q] != lb[q]) anti ^= 1;
        return anti == 0;
    };
    std::vector<std::vector<int64_t>> groups;
    for (int64_t t = 0; t < nt; ++t) {
        size_t g = 0;
        for (; g < groups.size(); ++g) {
            bool fits = true;
            for (int64_t s : groups[g])
                if (!commute(s, t)) { fits = false; break; }
            if (fits) break;
        }
        if (g == groups.size()) groups.emplace_back();
        groups[g].push_back(t);
        group[t] = (int32_t)g;
    }
    return (int64_t)groups.size();
}

}  // extern "C"

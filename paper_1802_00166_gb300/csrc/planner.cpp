#include "planner.h"

#include <algorithm>

namespace pcot {

namespace {

bool has_depth(const std::vector<int>& s, int d) {
    if (s.empty()) return d >= 1;
    return std::find(s.begin(), s.end(), d) != s.end();
}

int largest_leq(const std::vector<int>& s, int d) {
    if (s.empty()) return d;
    int best = 0;
    for (int v : s)
        if (v <= d && v > best) best = v;
    return best;
}

int64_t fdiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

struct Rec {
    int P, D, dims;
    int64_t L[3];
    int64_t theta[4];
    std::vector<int32_t>* out;
    LatticeOrderStats st;

    int32_t id(int64_t b, const int64_t* I) const {
        int64_t v = b;
        for (int a = 0; a < 3; ++a) v = v * L[a] + (a < dims ? I[a] : 0);
        return (int32_t)v;
    }

    // Block range of the orthant that meets the skewed lattice domain
    // { 0 <= b < P, b <= J_a <= b + L_a - 1 }; empty when lo > hi.
    void block_range(const int64_t* lo, const int64_t* sz, int64_t* blo, int64_t* bhi) const {
        int64_t l = std::max<int64_t>(lo[0], 0), h = std::min<int64_t>(lo[0] + sz[0] - 1, P - 1);
        for (int a = 0; a < dims; ++a) {
            const int64_t jl = lo[1 + a], jh = lo[1 + a] + sz[1 + a] - 1;
            l = std::max<int64_t>(l, jl - L[a] + 1);
            h = std::min<int64_t>(h, jh);
        }
        *blo = l;
        *bhi = h;
    }

    void leaf(const int64_t* lo, const int64_t* sz) {
        int64_t bl, bh;
        block_range(lo, sz, &bl, &bh);
        for (int64_t b = bl; b <= bh; ++b) {
            int64_t jl[3] = {0, 0, 0}, jh[3] = {0, 0, 0};
            bool any = true;
            for (int a = 0; a < dims; ++a) {
                jl[a] = std::max<int64_t>(lo[1 + a], b);
                jh[a] = std::min<int64_t>(lo[1 + a] + sz[1 + a] - 1, b + L[a] - 1);
                if (jl[a] > jh[a]) any = false;
            }
            if (!any) continue;
            int64_t J[3] = {jl[0], jl[1], jl[2]};
            for (;;) {
                int64_t I[3] = {0, 0, 0};
                for (int a = 0; a < dims; ++a) I[a] = J[a] - b;
                out->push_back(id(b, I));
                int a = dims - 1;
                for (; a >= 0; --a) {
                    if (++J[a] <= jh[a]) break;
                    J[a] = jl[a];
                }
                if (a < 0) break;
            }
        }
    }

    void go(const int64_t* lo, const int64_t* sz) {
        ++st.recursive_calls;
        for (int i = 0; i < D; ++i)
            if (sz[i] <= 0) {
                ++st.zero_exits;
                return;
            }
        int64_t bl, bh;
        block_range(lo, sz, &bl, &bh);
        if (bl > bh) {
            ++st.empty_exits;
            return;
        }
        bool base = true;
        for (int i = 0; i < D; ++i)
            if (sz[i] > theta[i]) base = false;
        if (base) {
            ++st.leaves;
            leaf(lo, sz);
            return;
        }
        for (int c = 0; c < (1 << D); ++c) {
            int64_t clo[4], csz[4];
            for (int i = 0; i < D; ++i) {
                const int bit = (c >> (D - 1 - i)) & 1;
                if (sz[i] > theta[i]) {
                    const int64_t h = sz[i] / 2;
                    clo[i] = lo[i] + (bit ? h : 0);
                    csz[i] = bit ? sz[i] - h : h;
                } else {
                    clo[i] = lo[i];
                    csz[i] = bit ? 0 : sz[i];
                }
            }
            go(clo, csz);
        }
    }
};

}  // namespace

BlockPlan plan_blocks(int64_t T, int k, const std::vector<int>& supported) {
    BlockPlan p;
    if (T <= 0) return p;
    if (k < 1) k = 1;
    if (!has_depth(supported, k)) k = std::max(1, largest_leq(supported, k));
    const int64_t main = T / k;
    for (int64_t i = 0; i < main; ++i) p.depths.push_back(k);
    int64_t rem = T - main * k;
    while (rem > 0) {
        const int d = std::max(1, largest_leq(supported, (int)std::min<int64_t>(rem, 1 << 20)));
        p.depths.push_back(d);
        rem -= d;
    }
    if (p.depths.size() % 2 == 1) {
        // Split the smallest block that splits into two supported depths.
        int best = -1;
        for (size_t i = 0; i < p.depths.size(); ++i) {
            const int d = p.depths[i];
            if (d < 2) continue;
            for (int a = 1; a < d; ++a)
                if (has_depth(supported, a) && has_depth(supported, d - a)) {
                    if (best < 0 || d < p.depths[best]) best = (int)i;
                    break;
                }
        }
        if (best >= 0) {
            const int d = p.depths[best];
            int a = 1;
            for (; a < d; ++a)
                if (has_depth(supported, a) && has_depth(supported, d - a)) break;
            p.depths[best] = d - a;
            p.depths.insert(p.depths.begin() + best + 1, a);
        } else {
            p.final_copy = true;
        }
    }
    return p;
}

std::vector<int32_t> pcot_lattice_order(int P, int dims, const int64_t* L, const int64_t* theta,
                                        LatticeOrderStats* stats) {
    std::vector<int32_t> out;
    if (P <= 0) return out;
    Rec r;
    r.P = P;
    r.D = dims + 1;
    r.dims = dims;
    for (int a = 0; a < 3; ++a) r.L[a] = a < dims ? L[a] : 1;
    for (int i = 0; i < 4; ++i) r.theta[i] = (i <= dims && theta && theta[i] > 0) ? theta[i] : 1;
    int64_t total = P;
    for (int a = 0; a < dims; ++a) total *= r.L[a];
    out.reserve((size_t)total);
    r.out = &out;
    // Bounding box of the skewed lattice, padded to theta * 2^k.
    int64_t lo[4] = {0, 0, 0, 0}, sz[4] = {P, 0, 0, 0};
    for (int a = 0; a < dims; ++a) sz[1 + a] = P + r.L[a] - 1;
    for (int i = 0; i < r.D; ++i) {
        int64_t s = r.theta[i];
        while (s < sz[i]) s *= 2;
        sz[i] = s;
    }
    r.go(lo, sz);
    if (stats) *stats = r.st;
    (void)fdiv;
    return out;
}

std::vector<int32_t> lattice_dep_counts(int P, int dims, const int64_t* L) {
    int64_t LL[3] = {1, 1, 1};
    for (int a = 0; a < dims; ++a) LL[a] = L[a];
    const int64_t per_block = LL[0] * LL[1] * LL[2];
    std::vector<int32_t> c((size_t)(P * per_block), 0);
    for (int64_t b = 1; b < P; ++b)
        for (int64_t i0 = 0; i0 < LL[0]; ++i0)
            for (int64_t i1 = 0; i1 < LL[1]; ++i1)
                for (int64_t i2 = 0; i2 < LL[2]; ++i2) {
                    auto span = [](int64_t i, int64_t n) {
                        return (int64_t)((i > 0) + 1 + (i + 1 < n));
                    };
                    const int64_t n = span(i0, LL[0]) * (dims > 1 ? span(i1, LL[1]) : 1) *
                                      (dims > 2 ? span(i2, LL[2]) : 1);
                    c[(size_t)(((b * LL[0] + i0) * LL[1] + i1) * LL[2] + i2)] = (int32_t)n;
                }
    return c;
}

}  // namespace pcot

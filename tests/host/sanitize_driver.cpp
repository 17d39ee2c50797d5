// Drives the host preprocessing (input cleaning, symmetry check, the three
// orderings, the classifier, relabelling) on awkward inputs so that a build
// with AddressSanitizer and UndefinedBehaviorSanitizer can check every path.
// Exit code 0 when every ordering is a permutation and every relabelled graph
// keeps its edge count; sanitizer reports abort the run by themselves.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "host_graph.h"

namespace {

uint64_t mix(uint64_t z) {   // SplitMix64 finaliser (Vigna), for test inputs only
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Raw, deliberately messy symmetric CSR: duplicates, self-loops, isolated vertices.
void make_graph(int32_t n, int64_t m, uint64_t seed, bool hubs, std::vector<int32_t>& rp, std::vector<int32_t>& ci) {
    std::vector<std::vector<int32_t>> adj((size_t)n);
    for (int64_t e = 0; e < m && n > 0; ++e) {
        const uint64_t a = mix(seed + 2 * (uint64_t)e + 1), b = mix(seed + 2 * (uint64_t)e + 2);
        int32_t u = (int32_t)(a % (uint64_t)n);
        int32_t v = (int32_t)(b % (uint64_t)n);
        if (hubs && (a & 3) == 0) u = (int32_t)(a % 3 % (uint64_t)n);   // a few heavy rows
        adj[(size_t)u].push_back(v);
        adj[(size_t)v].push_back(u);
        if ((b & 15) == 0) adj[(size_t)u].push_back(v);   // duplicate
    }
    rp.assign((size_t)n + 1, 0);
    ci.clear();
    for (int32_t u = 0; u < n; ++u) {
        for (int32_t v : adj[(size_t)u]) ci.push_back(v);
        rp[(size_t)u + 1] = (int32_t)ci.size();
    }
}

bool has_edge(const blest::Csr& g, int64_t u, int64_t v) {
    for (int64_t e = g.rp[(size_t)u]; e < g.rp[(size_t)u + 1]; ++e)
        if (g.ci[(size_t)e] == v) return true;
    return false;
}

// is_symmetric must reject g and name an edge (u, v) of g whose reverse is missing.
int expect_asymmetric(const blest::Csr& g, const char* what) {
    int64_t bu = -1, bv = -1;
    if (blest::is_symmetric(g, 2, &bu, &bv)) {
        std::printf("accepted asymmetric graph: %s\n", what);
        return 1;
    }
    if (bu < 0 || bv < 0 || bu >= g.n || bv >= g.n || !has_edge(g, bu, bv) || has_edge(g, bv, bu)) {
        std::printf("bad witness (%lld, %lld): %s\n", (long long)bu, (long long)bv, what);
        return 1;
    }
    return 0;
}

// g with one direction of one edge removed
blest::Csr drop_direction(const blest::Csr& g, int64_t u, int32_t v) {
    blest::Csr r;
    r.n = g.n;
    r.rp.assign((size_t)g.n + 1, 0);
    for (int32_t x = 0; x < g.n; ++x) {
        for (int64_t e = g.rp[(size_t)x]; e < g.rp[(size_t)x + 1]; ++e)
            if (!(x == u && g.ci[(size_t)e] == v)) r.ci.push_back(g.ci[(size_t)e]);
        r.rp[(size_t)x + 1] = (int32_t)r.ci.size();
    }
    return r;
}

bool is_perm(const std::vector<int32_t>& p, int32_t n) {
    if ((int32_t)p.size() != n) return false;
    std::vector<char> seen((size_t)n, 0);
    for (int32_t x : p) {
        if (x < 0 || x >= n || seen[(size_t)x]) return false;
        seen[(size_t)x] = 1;
    }
    return true;
}

}  // namespace

int main() {
    int failures = 0;
    const int32_t sizes[] = {0, 1, 2, 7, 9, 64, 333, 2048};
    for (int32_t n : sizes) {
        for (int hubs = 0; hubs < 2; ++hubs) {
            std::vector<int32_t> rp, ci;
            make_graph(n, 3 * (int64_t)n, 17 + (uint64_t)n, hubs != 0, rp, ci);
            blest::Csr g;
            std::string err;
            if (blest::clean_csr(n, rp.data(), ci.empty() ? nullptr : ci.data(), 2, g, err) != 0) {
                std::printf("clean_csr failed n=%d: %s\n", n, err.c_str());
                ++failures;
                continue;
            }
            int64_t bu = -1, bv = -1;
            if (!blest::is_symmetric(g, 2, &bu, &bv)) { std::printf("asymmetric n=%d\n", n); ++failures; }
            // one direction of a few edges removed, edges below and above the diagonal alike
            for (int64_t t = 0; t < 6 && g.nnz() > 0; ++t) {
                const int64_t e = (int64_t)(mix(99 + (uint64_t)n + 7 * (uint64_t)t) % (uint64_t)g.nnz());
                int64_t u = 0;
                while (g.rp[(size_t)u + 1] <= e) ++u;
                failures += expect_asymmetric(drop_direction(g, u, g.ci[(size_t)e]), "one direction dropped");
            }
            (void)blest::is_social_like(g);
            std::vector<int32_t> ids;
            blest::order_rcm(g, ids);
            failures += !is_perm(ids, n);
            blest::order_hub_prepass(g, ids);
            failures += !is_perm(ids, n);
            for (int32_t w : {8, 64, 4096}) {
                blest::order_jaccard_windows(g, 8, w, 3, ids);
                failures += !is_perm(ids, n);
                blest::order_compress(g, 8, w, 2, ids);
                failures += !is_perm(ids, n);
                blest::Csr r;
                blest::relabel_csr(g, ids, 2, r);
                failures += r.nnz() != g.nnz();
            }
        }
    }
    // RCM (its pseudo-peripheral search and its Cuthill-McKee levels) and the hub
    // pre-pass expand large levels on several threads: the order must not depend
    // on the thread count.  Levels of this graph exceed the parallel thresholds.
    {
        const int32_t n = 200000;
        std::vector<int32_t> rp, ci;
        make_graph(n, 8 * (int64_t)n, 4242, true, rp, ci);
        blest::Csr g;
        std::string err;
        if (blest::clean_csr(n, rp.data(), ci.data(), 4, g, err) != 0) {
            ++failures;
        } else {
            std::vector<int32_t> one, four;
            blest::order_rcm(g, one, 1);
            blest::order_rcm(g, four, 4);
            if (!is_perm(one, n) || one != four) { std::printf("RCM differs across thread counts\n"); ++failures; }
            blest::order_hub_prepass(g, one, 1);
            blest::order_hub_prepass(g, four, 4);
            if (!is_perm(one, n) || one != four) { std::printf("pre-pass differs across thread counts\n"); ++failures; }
            // relabelling sorts the long hub rows by radix: rows sorted, duplicate-free, edges kept
            blest::Csr r;
            blest::relabel_csr(g, four, 4, r);
            int64_t longest = 0;
            bool sorted = r.nnz() == g.nnz();
            for (int32_t u = 0; u < n && sorted; ++u) {
                longest = std::max<int64_t>(longest, r.rp[(size_t)u + 1] - r.rp[(size_t)u]);
                for (int64_t e = r.rp[(size_t)u] + 1; e < r.rp[(size_t)u + 1]; ++e)
                    if (r.ci[(size_t)e - 1] >= r.ci[(size_t)e]) sorted = false;
            }
            if (!sorted || longest <= 1024) { std::printf("relabelled rows: sorted %d longest %lld\n", sorted, (long long)longest); ++failures; }
        }
    }
    // a high-diameter layered graph: 120 layers of 1100 vertices, vertex i of a layer
    // joined to vertices 7i+3 and 11i+4 (mod 1100) of the next (one connected graph), so
    // that after a few levels a BFS level spans about a layer: 113 of its 122 levels
    // reach the size at which the FIFO levels of RCM and the pre-pass use the thread pool
    {
        const int32_t W = 1100, H = 120, n = W * H;
        std::vector<std::vector<int32_t>> adj((size_t)n);
        for (int32_t k = 0; k + 1 < H; ++k)
            for (int32_t i = 0; i < W; ++i) {
                const int32_t u = k * W + i;
                for (int32_t j : {(7 * i + 3) % W, (11 * i + 4) % W}) {
                    const int32_t v = (k + 1) * W + j;
                    adj[(size_t)u].push_back(v);
                    adj[(size_t)v].push_back(u);
                }
            }
        std::vector<int32_t> rp((size_t)n + 1, 0), ci;
        for (int32_t u = 0; u < n; ++u) {
            for (int32_t v : adj[(size_t)u]) ci.push_back(v);
            rp[(size_t)u + 1] = (int32_t)ci.size();
        }
        blest::Csr g;
        std::string err;
        if (blest::clean_csr(n, rp.data(), ci.data(), 4, g, err) != 0) {
            ++failures;
        } else {
            std::vector<int32_t> one, four;
            blest::order_rcm(g, one, 1);
            blest::order_rcm(g, four, 4);
            if (!is_perm(one, n) || one != four) { std::printf("layered RCM differs across thread counts\n"); ++failures; }
            blest::order_hub_prepass(g, one, 1);
            blest::order_hub_prepass(g, four, 4);
            if (!is_perm(one, n) || one != four) { std::printf("layered pre-pass differs across thread counts\n"); ++failures; }
        }
    }
    // a long row whose relabelled ids fill all three 10-bit radix digits (ids up to 2^23)
    {
        const int32_t n = 1 << 23, hub = 12345, deg = 5000;
        blest::Csr g;
        g.n = n;
        std::vector<int32_t> nb;
        for (int32_t i = 0; i < deg; ++i) nb.push_back((int32_t)(mix(777 + (uint64_t)i) % (uint64_t)n));
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        nb.erase(std::remove(nb.begin(), nb.end(), hub), nb.end());
        g.rp.assign((size_t)n + 1, 0);
        for (int32_t v = 0; v < n; ++v) g.rp[(size_t)v + 1] = g.rp[(size_t)v] + (v == hub ? (int32_t)nb.size() : 0);
        g.ci = nb;
        std::vector<int32_t> perm((size_t)n);
        for (int32_t v = 0; v < n; ++v) perm[(size_t)v] = v;
        for (int32_t v = n - 1; v > 0; --v) std::swap(perm[(size_t)v], perm[(size_t)(mix(31 + (uint64_t)v) % (uint64_t)(v + 1))]);
        blest::Csr r;
        blest::relabel_csr(g, perm, 2, r);
        std::vector<int32_t> expect;
        for (int32_t x : nb) expect.push_back(perm[(size_t)x]);
        std::sort(expect.begin(), expect.end());
        const int32_t w = perm[(size_t)hub];
        std::vector<int32_t> got(r.ci.begin() + r.rp[(size_t)w], r.ci.begin() + r.rp[(size_t)w + 1]);
        if (got != expect || expect.back() < (1 << 20)) { std::printf("radix row differs\n"); ++failures; }
    }
    // a lower edge without its reverse, next to a symmetric pair: only the edge count shows it
    {
        blest::Csr g;
        g.n = 4;
        g.rp = {0, 1, 2, 2, 3};   // 0-1 both ways, then 3 -> 1 alone
        g.ci = {1, 0, 1};
        failures += expect_asymmetric(g, "lower edge without reverse");
        blest::Csr h;
        h.n = 4;
        h.rp = {0, 1, 1, 1, 2};   // 0 -> 1 alone (upper) and 3 -> 2 alone (lower): equal counts
        h.ci = {1, 2};
        failures += expect_asymmetric(h, "upper and lower edges without reverse");
    }
    // invalid inputs are rejected, not read out of bounds
    {
        const int32_t rp[] = {0, 2, 1};
        const int32_t ci[] = {1, 0};
        blest::Csr g;
        std::string err;
        failures += blest::clean_csr(2, rp, ci, 1, g, err) == 0;
        const int32_t rp2[] = {0, 1, 2};
        const int32_t ci2[] = {5, 0};
        failures += blest::clean_csr(2, rp2, ci2, 1, g, err) == 0;
    }
    std::printf("failures=%d\n", failures);
    return failures == 0 ? 0 : 1;
}

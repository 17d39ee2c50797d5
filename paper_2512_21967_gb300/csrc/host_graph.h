// Host-side graph preprocessing: input validation and cleaning, the two vertex
// orderings of Section 3.2 (JaccardWithWindows with its pre-pass, and Reverse
// Cuthill-McKee), the social-like classifier of Section 3.2.1, and relabelling.
// Pure C++ (no CUDA); every routine is deterministic for a given input.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace blest {

struct Csr {
    int32_t n = 0;
    std::vector<int32_t> rp;   // n + 1
    std::vector<int32_t> ci;   // rp[n], rows sorted ascending, no duplicates, no self-loops
    int64_t nnz() const { return rp.empty() ? 0 : rp.back(); }
};

int host_threads(int requested);

// Validates (row_ptr[0] = 0, non-decreasing, ids in range) and cleans a raw CSR
// into `out`.  Returns 0 or a blest_status code; `err` gets a message.
int clean_csr(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int threads, Csr& out,
              std::string& err);

// true iff every (u, v) has (v, u).  Rows must be sorted (as after clean_csr).
bool is_symmetric(const Csr& g, int threads, int64_t* bad_u, int64_t* bad_v);

// Orderings; all return new_id[old].
// threads > 1: the BFS runs of the pseudo-peripheral search and large levels of
// the Cuthill-McKee pass are expanded in parallel (the same order).
void order_rcm(const Csr& g, std::vector<int32_t>& new_id, int threads = 1);
// threads > 1: large BFS levels are expanded in parallel (the same order).
void order_hub_prepass(const Csr& g, std::vector<int32_t>& new_id, int threads = 1);
// row_at (optional, n entries): window position p holds row row_at[p] of g
// (the identity when NULL); new_id is indexed by position.
void order_jaccard_windows(const Csr& g, int sigma, int32_t window, int threads,
                           std::vector<int32_t>& new_id, const int32_t* row_at = nullptr);
// Gorder (the pre-pass Section 3.2 names): window w, common neighbours of degree <= hub_cap.
void order_gorder(const Csr& g, int w, int32_t hub_cap, std::vector<int32_t>& new_id);
// The compression-oriented ordering: a pre-pass (0: BFS from the hubs, 1: Gorder with
// w = 5, hub_cap = 64), then JaccardWithWindows (Algorithm 1).
void order_compress(const Csr& g, int sigma, int32_t window, int threads, std::vector<int32_t>& new_id,
                    int prepass = 0);

// Section 3.2.1: heavy-tail sharing (top 1% of vertices by degree hold > 5% of
// the edges and top 10% hold > 40%) or a power-law-like log-log degree histogram.
bool is_social_like(const Csr& g);

// CSR of g with vertex v renamed new_id[v]; rows sorted.
void relabel_csr(const Csr& g, const std::vector<int32_t>& new_id, int threads, Csr& out);

}  // namespace blest

// Host-side preprocessing of HYLU (Sec. 2.1): static pivoting with scaling,
// fill-reducing ordering, symbolic factorization, supernode detection and the
// dependency schedule.  Runs once per sparsity pattern, before any numeric work.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace hylu {

struct CsrPattern {
    int32_t n = 0;
    std::vector<int64_t> rp;   // n+1
    std::vector<int32_t> ci;   // sorted within each row
};

// Maximum-product matching (Sec. 2.1, static pivoting [8]): row i is matched
// to column match_col[i]; dr/dc scale A so that matched entries have
// magnitude 1 and every entry magnitude <= 1.  Returns false when A is
// structurally singular (no perfect matching on its nonzero values).
bool max_product_matching(int32_t n, const int64_t* rp, const int32_t* ci, const double* v,
                          std::vector<int32_t>& match_col, std::vector<double>& dr,
                          std::vector<double>& dc);

// Approximate minimum degree ordering (Sec. 2.1 [9]) of a symmetric pattern
// given without its diagonal.  perm[k] = vertex eliminated k-th.
void amd_order(const CsrPattern& g, std::vector<int32_t>& perm, double dense_factor = 10.0);

// Nested dissection ordering (Sec. 2.1 [11]) of a symmetric pattern given
// without its diagonal; leaves of at most leaf_size vertices use AMD; vertices
// denser than max(16, dense_factor sqrt(n)) are ordered last, as in amd_order.
void nd_order(const CsrPattern& g, std::vector<int32_t>& perm, int32_t leaf_size = 256,
              double dense_factor = 2.0);

// Symmetric pattern of A + A^T without the diagonal, for an n x n CSR.
CsrPattern symmetrize(int32_t n, const int64_t* rp, const int32_t* ci);

}  // namespace hylu

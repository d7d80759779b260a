// Sparse products of a level's factor with the level transfers (host, FP64).
//
// The sweep carries every chain on the coarse side of both dimensions, so it
// applies a factor together with the transfer next to it: restriction after
// the factor (R_l X_{l+1}, rows on level l, columns on level l+1) and the
// factor after prolongation (X_l E_{l-1}, rows on level l, columns on level
// l-1).  Both follow from the Galerkin projection of Sect. 4.2 and the nested
// embeddings (E_{L<-l'} = E_{L<-l} E_{l<-l'}); they are formed once per level
// in FP64 and then rounded like every other factor value.
#include <algorithm>

#include "internal.h"

namespace sgdg {

Csr product_pattern(const Csr& A, const Csr& B) {
  Csr C;
  C.nrows = A.nrows;
  C.ncols = B.ncols;
  C.rowptr.assign(A.nrows + 1, 0);
  std::vector<int> mark(B.ncols, -1), cols;
  for (int i = 0; i < A.nrows; ++i) {
    cols.clear();
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
      const int k = A.col[p];
      for (int q = B.rowptr[k]; q < B.rowptr[k + 1]; ++q) {
        const int j = B.col[q];
        if (mark[j] != i) {
          mark[j] = i;
          cols.push_back(j);
        }
      }
    }
    std::sort(cols.begin(), cols.end());
    C.col.insert(C.col.end(), cols.begin(), cols.end());
    C.rowptr[i + 1] = (int)C.col.size();
  }
  return C;
}

void product_values(const Csr& A, const std::vector<double>& aval, const Csr& B, const std::vector<double>& bval,
                    const Csr& C, std::vector<double>& cval) {
  cval.assign(C.col.size(), 0.0);
  std::vector<int> pos(C.ncols, -1);
  for (int i = 0; i < A.nrows; ++i) {
    for (int r = C.rowptr[i]; r < C.rowptr[i + 1]; ++r) pos[C.col[r]] = r;
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
      const int k = A.col[p];
      const double a = aval[p];
      for (int q = B.rowptr[k]; q < B.rowptr[k + 1]; ++q) cval[pos[B.col[q]]] += a * bval[q];
    }
  }
}

}  // namespace sgdg

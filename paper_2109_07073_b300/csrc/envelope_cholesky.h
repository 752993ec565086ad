// Host-side envelope (skyline) Cholesky factorisation used by the pose solve.
#pragma once
#include <cstdint>

namespace vg {

// In place: a holds rows 0..n-1 of the lower envelope, row r's columns
// first[r]..r starting at a[off[r]]; n is a multiple of 6 and the six rows of
// each pose block share a first column that is a multiple of 6.  Returns false
// if the matrix is not positive definite (a pivot <= 0) or the layout is not
// of that form.
bool envelope_cholesky6(double *a, const int64_t *first, const int64_t *off, int64_t n);

}  // namespace vg

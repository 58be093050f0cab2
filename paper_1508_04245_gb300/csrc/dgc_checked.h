// Bounds checks of gather indices (neighbour codes, facet DOF ids, facet sides).
// Compiled in with -DDGC_CHECKED=1 (the test library libdgconv_checked.so): an
// index outside its range sets bit 3 of status[0], the first such index is kept
// in status[1], and the access is skipped (a neighbour counts as absent, a value
// reads as zero).  In the regular build the checks compile away.
#pragma once

#ifndef DGC_CHECKED
#define DGC_CHECKED 0
#endif

namespace dgc {

__device__ __forceinline__ bool gather_ok(long i, long n, int* status) {
#if DGC_CHECKED
  if (i >= 0 && i < n) return true;
  if (status && (atomicOr(status, 8) & 8) == 0)
    atomicExch(status + 1, (int)(i > 2147483647L ? 2147483647L : (i < -2147483647L ? -2147483647L : i)));
  return false;
#else
  (void)i;
  (void)n;
  (void)status;
  return true;
#endif
}

// a neighbour code (element << shift) | local facet, checked against E elements;
// an invalid one reads as -1 (no neighbour) in the checked build
__device__ __forceinline__ int checked_code(int code, int shift, long E, int* status) {
  return (code >= 0 && !gather_ok(code >> shift, E, status)) ? -1 : code;
}

}  // namespace dgc

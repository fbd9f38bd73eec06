// Temporary entry points for the low-rank drivers (replaced by rsvd.cu / nystrom.cu).
#include "common.cuh"

extern "C" {
int bsrht_rsvd(const void*, int64_t, int64_t, int32_t, int64_t, int32_t, uint64_t, double*, double*,
               double*, const bsrht_opts*) { return BSRHT_EUNSUP; }
int bsrht_rsvd_workspace(int64_t, int64_t, int32_t, int64_t, int32_t, const bsrht_opts*, size_t* b) {
  if (b) *b = 0;
  return BSRHT_EUNSUP;
}
int bsrht_nystrom(const void*, int64_t, int32_t, int64_t, int32_t, uint64_t, double*, double*,
                  const bsrht_opts*) { return BSRHT_EUNSUP; }
int bsrht_nystrom_workspace(int64_t, int32_t, int64_t, int32_t, const bsrht_opts*, size_t* b) {
  if (b) *b = 0;
  return BSRHT_EUNSUP;
}
}

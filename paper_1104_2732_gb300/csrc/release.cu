// Per-context resources of the subsystems beyond the single-array select.
#include "api_internal.h"

void gbs_internal_release(gbs_ctx* c) {
  gbs_internal_release_lms(c);
  gbs_internal_release_fused(c);
  gbs_internal_release_model(c);
  gbs_internal_release_knn(c);
  gbs_internal_release_search(c);
}

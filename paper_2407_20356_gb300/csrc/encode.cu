// placeholder, replaced by the tcgen05 encode
#include "internal.h"
extern "C" xpcs_status xpcs_encode(xpcs_ctx*, const xpcs_basis*, const void*, xpcs_dtype, int64_t, float*) {
  return XPCS_ENOTSUP;
}
extern "C" xpcs_status xpcs_fit_basis(xpcs_ctx*, const xpcs_rings*, const void*, xpcs_dtype, int64_t, int,
                                      xpcs_basis**, double*) {
  return XPCS_ENOTSUP;
}

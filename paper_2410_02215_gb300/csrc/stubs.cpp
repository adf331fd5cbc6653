// Entry points whose implementation is pending.
#include "common.h"

using namespace ftn;

extern "C" {

ftn_status ftn_contract(ftn_ctx, const ftn_network*, const ftn_tree*, ftn_prec, double*, double*) {
  return set_error(FTN_EUNSUPPORTED, "ftn_contract is not built yet");
}

ftn_status ftn_hubbard_term(ftn_ctx, int, double, double, ftn_dtype, ftn_tensor*) {
  return set_error(FTN_EUNSUPPORTED, "ftn_hubbard_term is not built yet");
}

}

// Release of batch and server objects; extended by the batching and serving units.
#include "hm_api_internal.h"

namespace hmi {

void destroy_other(void* any, uint32_t magic) {
  (void)any;
  (void)magic;
}

}  // namespace hmi

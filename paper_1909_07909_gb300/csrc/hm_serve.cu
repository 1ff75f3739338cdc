// Serving runtime (see include/hm.h).
#include "hm_api_internal.h"

namespace hmi {

void destroy_server(void* any) { (void)any; }

}  // namespace hmi

// SPSC and MPSC channels (HiCR paper Sec. 4.3, Channels frontend).
#include "hicr_internal.h"

namespace hicr {

struct Channel {};

void destroy_channels(Instance* in) {
  for (Channel* c : in->channels) delete c;
  in->channels.clear();
}

}  // namespace hicr

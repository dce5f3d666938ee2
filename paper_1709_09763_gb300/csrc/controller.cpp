// Host controller of the MLS^2MC sampler (Sec. 4.4): placeholder until the sampler lands.
#include "handle.h"

namespace mls2mc {

struct Sampler {};

int Handle::alloc_sampler() { return SMC_OK; }

void Handle::free_sampler() {
    delete smp;
    smp = nullptr;
}

}  // namespace mls2mc

// Learned merge scorer (placeholder: falls back to greedy).
#include "ajf_internal.h"

namespace ajf {

Path plan_learned(const Network& net, const PlanParams& p, uint64_t seed, bool* used) {
  if (used) *used = false;
  Path path = plan_greedy(net, p, seed, 0.0);
  return path;
}

}  // namespace ajf

// Admission policy of the request server (hz_server.cpp), kept free of CUDA
// so that it can be compiled and tested on its own.
//
// first_fit: the first queued request whose estimated device footprint fits
// in what the budget leaves (in_use + bytes <= budget), removed from the
// queue; null when none fits.  Every request ahead of the admitted one was
// passed over once more; a request passed over max_pass_over times stops the
// scan, so nothing behind it is admitted until it fits (large requests are
// not starved by a stream of small ones).
#pragma once

#include <cstdint>
#include <deque>

namespace hz {

template <class Request>
Request* first_fit(std::deque<Request*>& queue, uint64_t in_use, uint64_t budget, int max_pass_over) {
  for (auto it = queue.begin(); it != queue.end(); ++it) {
    Request* r = *it;
    if (in_use + r->bytes <= budget) {
      for (auto jt = queue.begin(); jt != it; ++jt) (*jt)->passed_over++;
      queue.erase(it);
      return r;
    }
    if (r->passed_over >= max_pass_over) return nullptr;
  }
  return nullptr;
}

}  // namespace hz

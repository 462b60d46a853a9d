// qp_host.cu -- host-side helper of the serving loop: many host-to-host copies in one call.
//
// The server packs each batch of requests into a pinned staging buffer (one slice per
// request and input) and unpacks the results the same way.  Done from Python, every small
// copy pays interpreter overhead under the interpreter lock; this call takes the whole list
// of (destination, source, size) triples and runs the copies on a few host threads.
#include <cstring>
#include <thread>
#include <vector>

#include "qp_gb300.h"

extern "C" int qp_host_copy_many(int count, void* const* dst, const void* const* src,
                                 const size_t* bytes, int threads) {
  if (count < 0 || (count > 0 && (!dst || !src || !bytes))) return QP_EINVAL;
  if (count == 0) return QP_OK;
  size_t total = 0;
  for (int i = 0; i < count; ++i) total += bytes[i];
  if (threads > 64) threads = 64;
  if (threads < 2 || total < (size_t(1) << 20)) {
    for (int i = 0; i < count; ++i)
      if (bytes[i]) std::memcpy(dst[i], src[i], bytes[i]);
    return QP_OK;
  }
  // Contiguous runs of copies of about total/threads bytes each.
  std::vector<int> cut(1, 0);
  size_t acc = 0;
  for (int i = 0; i < count && (int)cut.size() < threads; ++i) {
    acc += bytes[i];
    if (acc * threads >= total * cut.size()) cut.push_back(i + 1);
  }
  if (cut.back() != count) cut.push_back(count);
  std::vector<std::thread> pool;
  for (size_t t = 0; t + 1 < cut.size(); ++t) {
    const int i0 = cut[t], i1 = cut[t + 1];
    pool.emplace_back([=] {
      for (int i = i0; i < i1; ++i)
        if (bytes[i]) std::memcpy(dst[i], src[i], bytes[i]);
    });
  }
  for (auto& th : pool) th.join();
  return QP_OK;
}

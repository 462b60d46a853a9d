// qp_host.cu -- host-side helpers of the serving loop: many host-to-host copies in one call,
// and the gather/scatter of a packed batch's per-instance host arrays.
//
// The server packs each batch of requests into a pinned staging buffer (one slice per
// request and input) and unpacks the results the same way.  Done from Python, every small
// copy pays interpreter overhead under the interpreter lock; these calls take the whole
// batch and run the copies on a few host threads.
#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "qp_gb300.h"

namespace {

// Runs body(i) for i < count on up to `threads` host threads, in contiguous ranges of about
// equal weight (weight(i) bytes each).
template <typename W, typename F>
void run_split(int count, int threads, W weight, F body) {
  size_t total = 0;
  for (int i = 0; i < count; ++i) total += weight(i);
  if (threads > 64) threads = 64;
  if (threads < 2 || total < (size_t(1) << 20)) {
    for (int i = 0; i < count; ++i) body(i);
    return;
  }
  std::vector<int> cut(1, 0);
  size_t acc = 0;
  for (int i = 0; i < count && (int)cut.size() < threads; ++i) {
    acc += weight(i);
    if (acc * threads >= total * cut.size()) cut.push_back(i + 1);
  }
  if (cut.back() != count) cut.push_back(count);
  std::vector<std::thread> pool;
  for (size_t t = 0; t + 1 < cut.size(); ++t) {
    const int i0 = cut[t], i1 = cut[t + 1];
    pool.emplace_back([=] {
      for (int i = i0; i < i1; ++i) body(i);
    });
  }
  for (auto& th : pool) th.join();
}

// Elements and packed offset of field `rule` (QP_FIELD_*) of one instance.
bool field_of(const qp_instance_desc& d, int rule, int64_t* len, int64_t* off) {
  const int64_t n = d.n, p = d.nineq, m = d.neq;
  switch (rule) {
    case QP_FIELD_Q: *len = n * n; *off = d.oQ; return true;
    case QP_FIELD_Q1: *len = n; *off = d.oq; return true;
    case QP_FIELD_G: *len = p * n; *off = d.oG; return true;
    case QP_FIELD_H: *len = p; *off = d.oh; return true;
    case QP_FIELD_A: *len = m * n; *off = d.oA; return true;
    case QP_FIELD_B: *len = m; *off = d.ob; return true;
    default: return false;
  }
}

}  // namespace

extern "C" int qp_host_copy_many(int count, void* const* dst, const void* const* src,
                                 const size_t* bytes, int threads) {
  if (count < 0 || (count > 0 && (!dst || !src || !bytes))) return QP_EINVAL;
  if (count == 0) return QP_OK;
  run_split(count, threads, [&](int i) { return bytes[i]; },
            [&](int i) {
              if (bytes[i]) std::memcpy(dst[i], src[i], bytes[i]);
            });
  return QP_OK;
}

extern "C" int qp_host_pack(int B, const qp_instance_desc* desc, int esz, int nfields,
                            const int32_t* fields, const int64_t* sec, const void* const* src,
                            void* dst, int threads) {
  if (B < 0 || nfields < 0 || (esz != 4 && esz != 8)) return QP_EINVAL;
  if (B == 0 || nfields == 0) return QP_OK;
  if (!desc || !fields || !sec || !src || !dst) return QP_EINVAL;
  int64_t len, off;
  for (int f = 0; f < nfields; ++f)
    if (!field_of(desc[0], fields[f], &len, &off)) return QP_EINVAL;
  for (int k = 0; k < B; ++k)
    if (desc[k].id < 0 || desc[k].id >= B) return QP_EINVAL;
  char* out = static_cast<char*>(dst);
  run_split(B, threads,
            [&](int k) {
              const qp_instance_desc& d = desc[k];
              return (size_t)esz * (size_t)(d.n * (int64_t)(d.n + d.nineq + d.neq + 2) + d.nineq + d.neq);
            },
            [&](int k) {
              const qp_instance_desc& d = desc[k];
              for (int f = 0; f < nfields; ++f) {
                int64_t l, o;
                field_of(d, fields[f], &l, &o);
                const void* s = src[(size_t)d.id * nfields + f];
                if (l > 0 && s) std::memcpy(out + (size_t)(sec[f] + o) * esz, s, (size_t)l * esz);
              }
            });
  return QP_OK;
}

extern "C" int qp_host_unpack(int B, const qp_instance_desc* desc, int esz, int nfields,
                              const int32_t* fields, const int64_t* sec, const void* src,
                              void* dst, int64_t* dst_off, int threads) {
  if (B < 0 || nfields < 0 || (esz != 4 && esz != 8)) return QP_EINVAL;
  if (B == 0) return QP_OK;
  if (!desc || !fields || !sec || !src || !dst || !dst_off) return QP_EINVAL;
  int64_t len, off;
  for (int f = 0; f < nfields; ++f)
    if (!field_of(desc[0], fields[f], &len, &off)) return QP_EINVAL;
  // Instance id's fields land contiguously, in field order, at dst_off[id] elements.
  std::vector<const qp_instance_desc*> by_id(B, nullptr);
  for (int k = 0; k < B; ++k) {
    if (desc[k].id < 0 || desc[k].id >= B || by_id[desc[k].id]) return QP_EINVAL;
    by_id[desc[k].id] = &desc[k];
  }
  int64_t acc = 0;
  for (int i = 0; i < B; ++i) {
    dst_off[i] = acc;
    for (int f = 0; f < nfields; ++f) {
      field_of(*by_id[i], fields[f], &len, &off);
      acc += len;
    }
  }
  dst_off[B] = acc;
  const char* in = static_cast<const char*>(src);
  char* out = static_cast<char*>(dst);
  run_split(B, threads,
            [&](int i) { return (size_t)esz * (size_t)(dst_off[i + 1] - dst_off[i]); },
            [&](int i) {
              int64_t o = dst_off[i];
              for (int f = 0; f < nfields; ++f) {
                int64_t l, so;
                field_of(*by_id[i], fields[f], &l, &so);
                if (l > 0) std::memcpy(out + (size_t)o * esz, in + (size_t)(sec[f] + so) * esz, (size_t)l * esz);
                o += l;
              }
            });
  return QP_OK;
}

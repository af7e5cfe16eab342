// Data Object frontend (HiCR paper Sec. 4.3): publish / getHandle / get on top
// of the communication manager's memcpy.
#include <map>
#include <mutex>

#include "../../include/hicr_dataobject.h"
#include "hicr_internal.h"

namespace hicr {

struct DataObject {
  hicr_slot_t slot;
  uint64_t off, n;
};

struct DobjTable {
  uint64_t next = 1;
  std::map<uint64_t, DataObject> objs;
};

// per-instance tables (an instance is used by one host thread at a time)
static std::mutex g_dobj_mutex;
static std::map<const Instance*, DobjTable> g_dobj;

static DobjTable& table(const Instance* in) {
  std::lock_guard<std::mutex> lock(g_dobj_mutex);
  return g_dobj[in];
}

void forget_data_objects(const Instance* in) {
  std::lock_guard<std::mutex> lock(g_dobj_mutex);
  g_dobj.erase(in);
}

}  // namespace hicr

using namespace hicr;

extern "C" {

hicr_status hicr_dobj_publish(hicr_instance_t h, hicr_slot_t slot, uint64_t off, uint64_t n, uint64_t* id) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || !id) return HICR_ERR_INVALID;
  uint64_t size = 0;
  if (hicr_slot_info(h, slot, nullptr, &size, nullptr, nullptr) != HICR_OK) return HICR_ERR_INVALID;
  if (off > size || n > size - off) return HICR_ERR_BOUNDS;
  DobjTable& t = table(in);
  const uint64_t k = t.next++;
  t.objs[k] = DataObject{slot, off, n};
  *id = k;
  return HICR_OK;
}

hicr_status hicr_dobj_get_handle(hicr_instance_t h, uint64_t id, hicr_dobj_handle_t* out) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || !out) return HICR_ERR_INVALID;
  DobjTable& t = table(in);
  auto it = t.objs.find(id);
  if (it == t.objs.end()) return HICR_ERR_INVALID;
  uint32_t space = 0;
  if (hicr_slot_info(h, it->second.slot, nullptr, nullptr, &space, nullptr) != HICR_OK) return HICR_ERR_INVALID;
  out->id = id;
  out->size = it->second.n;
  out->space = space;
  out->instance = 0;
  return HICR_OK;
}

hicr_status hicr_dobj_get(hicr_instance_t h, const hicr_dobj_handle_t* handle, hicr_slot_t dst, uint64_t dst_off) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || !handle || handle->instance != 0) return HICR_ERR_INVALID;
  DobjTable& t = table(in);
  auto it = t.objs.find(handle->id);
  if (it == t.objs.end()) return HICR_ERR_INVALID;
  const DataObject o = it->second;
  return hicr_memcpy(h, dst, dst_off, o.slot, o.off, o.n);
}

hicr_status hicr_dobj_release(hicr_instance_t h, uint64_t id) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in) return HICR_ERR_INVALID;
  DobjTable& t = table(in);
  return t.objs.erase(id) ? HICR_OK : HICR_ERR_INVALID;
}

}  // extern "C"

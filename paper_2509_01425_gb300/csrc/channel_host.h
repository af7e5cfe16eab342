// Host side of the channels, shared by the channel host calls
// (channels.cu), the streaming runs (streams.cu) and the ping-pong
// (pingpong.cu): the channel record, handle lookup, the instance's reusable
// device buffer for launch arguments and results, and the device views of a
// channel.
#pragma once

#include <vector>

#include "channel_common.cuh"
#include "hicr_internal.h"

namespace hicr {

struct Channel {
  int kind = 0;  // 0 SPSC, 1 MPSC (locking), 2 MPSC (non-locking)
  bool live = false;
  uint32_t token_size = 0, capacity = 0;
  uint32_t n_producers = 0, max_msgs = 0;
  uint64_t ring_bytes = 0;
  uint8_t* ring = nullptr;
  void* state = nullptr;
  MpscMeta* meta = nullptr;
  hicr_slot_t ring_slot = 0;
  std::vector<uint32_t> seq;  // host-API producers' next sequence numbers
};

inline Channel* get(Instance* in, hicr_channel_t ch) {
  if (ch >= in->channels.size() || !in->channels[ch] || !in->channels[ch]->live) return nullptr;
  return in->channels[ch];
}

inline hicr_status dev_buffer(Instance* in, size_t bytes, void** out) {
  if (in->chan_buf_cap < bytes) {
    HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
    if (in->chan_buf) cudaFree(in->chan_buf);
    in->chan_buf = nullptr;
    in->chan_buf_cap = 0;
    size_t cap = bytes < 65536 ? 65536 : bytes;
    HICR_CUDA(in, cudaMalloc(&in->chan_buf, cap));
    in->chan_buf_cap = cap;
  }
  *out = in->chan_buf;
  return HICR_OK;
}

inline SpscView spsc_view(Channel* c) {
  SpscView v;
  v.ring = c->ring;
  v.st = (SpscState*)c->state;
  v.ts = c->token_size;
  v.cap = c->capacity;
  return v;
}
inline MpscView mpsc_view(Channel* c) {
  MpscView v;
  v.ring = c->ring;
  v.st = (MpscState*)c->state;
  v.meta = c->meta;
  v.R = c->ring_bytes;
  v.M = c->max_msgs;
  return v;
}

inline NlView nl_view(Channel* c) {
  NlView v;
  v.ring = c->ring;
  v.head = (NlHead*)c->state;
  v.st = (NlState*)((char*)c->state + sizeof(NlHead));
  v.meta = reinterpret_cast<NlMeta*>(c->meta);
  v.R = c->ring_bytes;
  v.M = c->max_msgs;
  v.P = c->n_producers;
  return v;
}

}  // namespace hicr

inline hicr::Instance* I(hicr_instance_t h) { return h ? &h->impl : nullptr; }

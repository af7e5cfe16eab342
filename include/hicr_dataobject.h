/*
 * hicr_dataobject.h -- Data Object frontend of libhicr_gb300.so.
 *
 * HiCR paper Sec. 4.3 (Built-in Frontends, Data Object): a data object is a
 * block of data inside a local memory slot made accessible by `publish`,
 * which returns a unique identifier; `getHandle` turns an identifier into a
 * handle (the metadata needed to fetch the object) and `get` starts an
 * asynchronous transfer of the object whose completion is fenced like any
 * memcpy (Fig. 5). With one instance the transfer is a local-to-local copy on
 * the communication stream.
 *
 * Conventions as in hicr.h.
 */
#ifndef HICR_DATAOBJECT_H
#define HICR_DATAOBJECT_H

#include <stdint.h>

#include "hicr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint64_t id;       /* identifier returned by publish (>= 1) */
  uint64_t size;     /* object bytes */
  uint32_t space;    /* memory space holding the object */
  uint32_t instance; /* owning instance (0: the only one) */
} hicr_dobj_handle_t;

/* Publish bytes [off, off+n) of `slot` as a data object; *id receives a new
 * identifier (1, 2, ... in publication order). The slot must stay live while
 * the object is published. Errors: INVALID (dead slot), BOUNDS. */
hicr_status hicr_dobj_publish(hicr_instance_t inst, hicr_slot_t slot, uint64_t off, uint64_t n, uint64_t* id);

/* The handle of a published object. Errors: INVALID (unknown identifier). */
hicr_status hicr_dobj_get_handle(hicr_instance_t inst, uint64_t id, hicr_dobj_handle_t* out);

/* Start copying the object into `dst` at dst_off (asynchronous; complete
 * after a fence of the destination's tag). Errors: INVALID (unknown object or
 * slot), BOUNDS, UNSUPPORTED (space pair), OVERLAP (object and destination
 * ranges intersect in one slot). */
hicr_status hicr_dobj_get(hicr_instance_t inst, const hicr_dobj_handle_t* handle, hicr_slot_t dst,
                          uint64_t dst_off);

/* Withdraw a published object; its identifier is not reused. Errors: INVALID. */
hicr_status hicr_dobj_release(hicr_instance_t inst, uint64_t id);

#ifdef __cplusplus
}
#endif

#endif /* HICR_DATAOBJECT_H */

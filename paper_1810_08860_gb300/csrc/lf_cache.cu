// lf_cache.cu - the host-side page cache of streamed light field images
// (the tile cache of Sec. 4.2.1 and the per-frame decode budget of the
// two-level progressive renderer, Sec. 7.2).  Pure host code: it decides which
// items (images) occupy which of a fixed number of device pages; the caller
// copies the admitted items into their pages.  No CUDA calls.
//
// Per frame the caller lists the items the frame wants, most important first.
// Resident wanted items stay.  Missing ones are admitted in list order, at
// most `budget` of them, each into a free page or else into the page of the
// oldest admitted item the frame does not want (first in, first out, as the
// paper's cache evicts).  Wanted items that find no page stay missing: the
// renderer draws the coarse level in their place.
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/lf.h"

struct lf_cache {
  int32_t n_items = 0, capacity = 0;
  std::vector<int32_t> page_of;   // item -> page, -1 when not resident
  std::vector<int32_t> item_in;   // page -> item, -1 when free
  std::vector<int64_t> admitted;  // page -> admission number (FIFO order)
  int64_t clock = 0;
  std::vector<int64_t> wanted_mark;  // item -> frame number that last wanted it
  int64_t frame = 0;
};

extern "C" {

lf_status lf_cache_create(int32_t n_items, int32_t capacity, lf_cache** out) {
  if (!out) return LF_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_items < 1 || capacity < 1) return LF_ERR_INVALID_ARG;
  lf_cache* c = new (std::nothrow) lf_cache();
  if (!c) return LF_ERR_OOM;
  try {
    c->n_items = n_items;
    c->capacity = capacity;
    c->page_of.assign(n_items, -1);
    c->item_in.assign(capacity, -1);
    c->admitted.assign(capacity, -1);
    c->wanted_mark.assign(n_items, -1);
  } catch (...) {
    delete c;
    return LF_ERR_OOM;
  }
  *out = c;
  return LF_OK;
}

void lf_cache_destroy(lf_cache* c) { delete c; }

lf_status lf_cache_frame(lf_cache* c, int32_t n_wanted, const int32_t* wanted, int32_t budget,
                         int32_t* n_uploads, int32_t* upload_items, int32_t* upload_pages) {
  if (!c || n_wanted < 0 || budget < 0 || !n_uploads || (n_wanted > 0 && !wanted)) return LF_ERR_INVALID_ARG;
  if (budget > 0 && (!upload_items || !upload_pages)) return LF_ERR_INVALID_ARG;
  for (int32_t k = 0; k < n_wanted; ++k)
    if (wanted[k] < 0 || wanted[k] >= c->n_items) return LF_ERR_INVALID_ARG;
  const int64_t f = ++c->frame;
  for (int32_t k = 0; k < n_wanted; ++k) c->wanted_mark[wanted[k]] = f;
  int32_t n = 0;
  for (int32_t k = 0; k < n_wanted && n < budget; ++k) {
    const int32_t item = wanted[k];
    if (c->page_of[item] >= 0) continue;  // resident (or admitted earlier in this list)
    int32_t page = -1;
    int64_t oldest = INT64_MAX;
    for (int32_t p = 0; p < c->capacity; ++p) {
      const int32_t it = c->item_in[p];
      if (it < 0) { page = p; break; }                 // a free page first
      if (c->wanted_mark[it] == f) continue;           // this frame needs it
      if (c->admitted[p] < oldest) { oldest = c->admitted[p]; page = p; }
    }
    if (page < 0) break;  // every page holds an item this frame wants
    if (c->item_in[page] >= 0) c->page_of[c->item_in[page]] = -1;
    c->item_in[page] = item;
    c->page_of[item] = page;
    c->admitted[page] = c->clock++;
    upload_items[n] = item;
    upload_pages[n] = page;
    ++n;
  }
  *n_uploads = n;
  return LF_OK;
}

lf_status lf_cache_pages(const lf_cache* c, int32_t* page_of_item) {
  if (!c || !page_of_item) return LF_ERR_INVALID_ARG;
  for (int32_t i = 0; i < c->n_items; ++i) page_of_item[i] = c->page_of[i];
  return LF_OK;
}

}  // extern "C"

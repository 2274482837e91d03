// psc_readout.h -- device-side read-out of a molecule list in id order.
#pragma once
#include "psc_internal.h"

namespace psc {

// The first n entries of `list` in ascending id order: out[3a..3a+2] their
// (i, j, k), or with `unwrapped` their unwrapped (X, Y, Z) (HCP or FCC
// basis, psc.h), and out_ids[a] their ids.  keys and slots hold n words each,
// scratch sorts n pairs; out (3n words) and out_ids (n words) are device
// buffers.  Ids must be distinct.  0 on success, a negative value when the
// sort does not fit its scratch or a launch failed.
int readout_positions(const SpeciesList& list, int32_t n, int32_t ni, int32_t nj, int32_t nk, bool unwrapped,
                      bool fcc, uint32_t* keys, uint32_t* slots, SortScratch& scratch, int32_t* out,
                      uint32_t* out_ids, int blocks, cudaStream_t st, int64_t* launches);

}  // namespace psc

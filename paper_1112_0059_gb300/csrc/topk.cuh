// Per-row bounded max-heap of neighbour keys (the k+1 nearest of Alg. 2).
// One thread owns one heap; the heap lives in memory (global or shared) so
// that k up to LNBNN_MAX_K needs no registers.
#pragma once

#include "internal.cuh"

namespace lnbnn {

// Max-heap of at most `cap` keys at h[0..cap).  Keys are distinct (each holds a
// distinct reference row), so no two compare equal.
struct TopK {
  uint64_t* h;
  int cap;
  int size;
  // Distance of the current largest key (INT32_MAX until the heap is full).
  // When keys arrive in increasing row order, only distances strictly below
  // it can enter; push() itself compares full (distance, row) keys.
  int32_t threshold;

  __device__ __forceinline__ TopK(uint64_t* heap, int K1) : h(heap), cap(K1), size(0), threshold(INT32_MAX) {}

  __device__ __forceinline__ void sift_down_root(uint64_t key, int n) {
    int i = 0;
    for (;;) {
      const int l = 2 * i + 1;
      if (l >= n) break;
      const int r = l + 1;
      uint64_t cv = h[l];
      int c = l;
      if (r < n) {
        const uint64_t rv = h[r];
        if (rv > cv) {
          cv = rv;
          c = r;
        }
      }
      if (cv <= key) break;
      h[i] = cv;
      i = c;
    }
    h[i] = key;
  }

  // Offer one key; keeps the `cap` smallest keys seen.
  __device__ __forceinline__ void push(uint64_t key) {
    if (size < cap) {
      int i = size++;
      while (i > 0) {
        const int p = (i - 1) >> 1;
        const uint64_t pv = h[p];
        if (pv >= key) break;
        h[i] = pv;
        i = p;
      }
      h[i] = key;
      if (size == cap) threshold = (int32_t)key_dist(h[0]);
    } else if (key < h[0]) {
      sift_down_root(key, cap);
      threshold = (int32_t)key_dist(h[0]);
    }
  }

  // Sort the kept keys ascending in place; unused slots become kEmptyKey.
  __device__ __forceinline__ void finish() {
    for (int end = size - 1; end > 0; --end) {
      const uint64_t top = h[0];
      const uint64_t last = h[end];
      h[end] = top;
      sift_down_root(last, end);
    }
    for (int i = size; i < cap; ++i) h[i] = kEmptyKey;
  }
};

}  // namespace lnbnn

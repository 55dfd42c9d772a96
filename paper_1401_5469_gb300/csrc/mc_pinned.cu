// Pinned host blocks reused across models and batches.
//
// cudaHostAlloc and cudaFreeHost synchronise the whole device, so a model or
// batch created or destroyed while other models' iterations run on their own
// streams would wait for all of them.  Blocks handed back here are kept and
// handed out again (by size class, mapped or not) instead of being freed; the
// cache holds at most the peak number of blocks in use at one time, until the
// process exits.
#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "mc_model_internal.h"

namespace mcgpu {

namespace {

struct Block {
  size_t cls;
  bool mapped;
};

std::mutex g_lock;
std::unordered_map<void *, Block> g_blocks;            // every block handed out, by address
std::unordered_map<uint64_t, std::vector<void *>> g_free;  // (class, mapped) -> free blocks

size_t size_class(size_t bytes) {
  size_t c = 64;
  while (c < bytes) c <<= 1;
  return c;
}

uint64_t key(size_t cls, bool mapped) { return (static_cast<uint64_t>(cls) << 1) | (mapped ? 1u : 0u); }

}  // namespace

void *pinned_get(size_t bytes, bool mapped) {
  const size_t cls = size_class(bytes);
  std::lock_guard<std::mutex> lk(g_lock);
  std::vector<void *> &fl = g_free[key(cls, mapped)];
  if (!fl.empty()) {
    void *p = fl.back();
    fl.pop_back();
    return p;
  }
  void *p = nullptr;
  if (cudaHostAlloc(&p, cls, mapped ? cudaHostAllocMapped : cudaHostAllocDefault) != cudaSuccess) return nullptr;
  g_blocks[p] = Block{cls, mapped};
  return p;
}

void pinned_put(void *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_lock);
  const auto it = g_blocks.find(p);
  if (it == g_blocks.end()) return;
  g_free[key(it->second.cls, it->second.mapped)].push_back(p);
}

}  // namespace mcgpu

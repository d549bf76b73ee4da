// wsm_arena.h -- the bookkeeping of the server's device arena: first-fit
// placement over [0, capacity) in 256-byte granules, with neighbouring free
// ranges merged on release.  Plain C++ (no CUDA): the server owns the device
// allocation the offsets index into.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace wsm {

class ArenaBook {
  public:
    static constexpr size_t kGranule = 256;
    static size_t round_up(size_t b) { return (b + kGranule - 1) & ~(kGranule - 1); }

    // Forget every block: one free range of `bytes` rounded up to a granule.
    void reset(size_t bytes) {
        capacity_ = round_up(bytes);
        used_ = 0;
        free_.clear();
        if (capacity_) free_[0] = capacity_;
    }
    size_t capacity() const { return capacity_; }
    size_t used() const { return used_; }
    // offset -> size of every free range, ascending, never two adjacent
    const std::map<size_t, size_t>& free_ranges() const { return free_; }

    // Offset of the lowest free range that holds `bytes` (rounded up), now
    // taken; SIZE_MAX if none does.
    size_t alloc(size_t bytes) {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, left = it->second - bytes;
            free_.erase(it);
            if (left) free_[off + bytes] = left;
            used_ += bytes;
            return off;
        }
        return SIZE_MAX;
    }

    // Return the block at `off` of `bytes` (as passed to alloc), merging it
    // with the free ranges right after and right before it.
    void release(size_t off, size_t bytes) {
        bytes = round_up(bytes);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }

  private:
    size_t capacity_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;   // offset -> size
};

}  // namespace wsm

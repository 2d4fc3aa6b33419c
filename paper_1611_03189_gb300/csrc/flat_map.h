// Open-addressing hash map from 64-bit keys (linear probing, power-of-two
// capacity, tombstones for erased keys), iterated in slot order.  The host
// side of the factorization looks up and inserts some hundred thousand
// blocks per refactor of a 512 x 512 problem; a node-based map spent a large
// part of the host's time in allocation and pointer chasing there.
//
// Iteration order depends only on the sequence of inserts and erases, so it
// is the same on every run.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <utility>
#include <vector>

namespace hs {

template <typename V>
class FlatMap {
 public:
  struct Slot {
    uint64_t first;
    V second;
  };

  class iterator {
   public:
    iterator(FlatMap *m, size_t i) : m_(m), i_(i) { skip(); }
    Slot &operator*() const { return m_->slots_[i_]; }
    Slot *operator->() const { return &m_->slots_[i_]; }
    iterator &operator++() {
      ++i_;
      skip();
      return *this;
    }
    bool operator==(const iterator &o) const { return i_ == o.i_; }
    bool operator!=(const iterator &o) const { return i_ != o.i_; }

   private:
    void skip() {
      while (i_ < m_->state_.size() && m_->state_[i_] != kFull) ++i_;
    }
    FlatMap *m_;
    size_t i_;
  };

  FlatMap() { init(16); }

  // room for n keys without growing
  void reserve(size_t n) {
    size_t c = 16;
    while (c * 7 < (n + 1) * 10) c <<= 1;
    if (c > state_.size()) rehash(c);
  }

  size_t size() const { return size_; }

  iterator begin() { return iterator(this, 0); }
  iterator end() { return iterator(this, state_.size()); }

  iterator find(uint64_t k) {
    const size_t i = locate(k);
    return i == kNone ? end() : iterator(this, i);
  }
  size_t count(uint64_t k) const { return locate(k) == kNone ? 0 : 1; }

  // the value of k, inserted value-initialised when missing; second: inserted
  // (a lookup of a present key never rehashes; an insert may, which moves
  // every value: references into the map do not survive an insert)
  std::pair<V *, bool> try_emplace(uint64_t k) {
    const size_t at = locate(k);
    if (at != kNone) return {&slots_[at].second, false};
    if ((size_ + tombs_ + 1) * 10 > state_.size() * 7) rehash(size_ * 10 > state_.size() * 4 ? 2 * state_.size()
                                                                                           : state_.size());
    const size_t mask = state_.size() - 1;
    size_t i = hash(k) & mask, tomb = kNone;
    while (true) {
      if (state_[i] == kEmpty) break;
      if (state_[i] == kFull && slots_[i].first == k) return {&slots_[i].second, false};
      if (state_[i] == kTomb && tomb == kNone) tomb = i;
      i = (i + 1) & mask;
    }
    if (tomb != kNone) {
      i = tomb;
      --tombs_;
    }
    state_[i] = kFull;
    slots_[i].first = k;
    slots_[i].second = V();
    ++size_;
    return {&slots_[i].second, true};
  }
  V &operator[](uint64_t k) { return *try_emplace(k).first; }

  void erase(uint64_t k) {
    const size_t i = locate(k);
    if (i == kNone) return;
    state_[i] = kTomb;
    --size_;
    ++tombs_;
  }

  void clear() { init(16); }

  void swap(FlatMap &o) {
    slots_.swap(o.slots_);
    state_.swap(o.state_);
    std::swap(size_, o.size_);
    std::swap(tombs_, o.tombs_);
  }

 private:
  static constexpr uint8_t kEmpty = 0, kFull = 1, kTomb = 2;
  static constexpr size_t kNone = ~(size_t)0;

  static uint64_t hash(uint64_t x) {   // the splitmix64 finaliser
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
  }

  size_t locate(uint64_t k) const {
    const size_t mask = state_.size() - 1;
    size_t i = hash(k) & mask;
    while (state_[i] != kEmpty) {
      if (state_[i] == kFull && slots_[i].first == k) return i;
      i = (i + 1) & mask;
    }
    return kNone;
  }

  void init(size_t cap) {
    slots_.assign(cap, Slot{0, V()});
    state_.assign(cap, kEmpty);
    size_ = tombs_ = 0;
  }

  // re-inserts the keys in slot order (deterministic)
  void rehash(size_t cap) {
    std::vector<Slot> old_slots;
    std::vector<uint8_t> old_state;
    old_slots.swap(slots_);
    old_state.swap(state_);
    init(cap);
    const size_t mask = cap - 1;
    for (size_t j = 0; j < old_state.size(); ++j) {
      if (old_state[j] != kFull) continue;
      size_t i = hash(old_slots[j].first) & mask;
      while (state_[i] != kEmpty) i = (i + 1) & mask;
      state_[i] = kFull;
      slots_[i] = old_slots[j];
      ++size_;
    }
  }

  std::vector<Slot> slots_;
  std::vector<uint8_t> state_;
  size_t size_ = 0, tombs_ = 0;
};

}  // namespace hs

// sft_slots.h -- capacity of the per-bin solution slots.
#pragma once

namespace sft {
// Recovered frequencies are filed under their level-0 bin k0 = s mod M0; a
// level-0 bin holds at most a_max <= 8 of them (a bin with more aliases is
// never solved), so 8 slots per bin never overflow.
constexpr int kSlots = 8;
}  // namespace sft

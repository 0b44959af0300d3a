// Host-side reference: named contigs concatenated into the index's text,
// ambiguous bytes replaced and recorded.  Shared by reference.cpp (building,
// persisting, filtering) and sam.cpp (SAM records).  No CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "mica.h"

struct mica_reference {
    std::vector<std::string> names;
    std::vector<uint64_t> start;     // n_contigs + 1 bounds: contig i = [start[i], start[i + 1])
    std::vector<uint64_t> amb_start; // maximal ambiguous runs [amb_start[j], amb_end[j]), ascending
    std::vector<uint64_t> amb_end;
    std::vector<uint8_t> text;       // G as 'A','C','G','T'
};

namespace mica {

constexpr int32_t PLACE_OFF_REFERENCE = -1;  // across a contig boundary or over an ambiguous base
constexpr int32_t PLACE_OUT_OF_RANGE = -2;   // the window ends past G (bad input)

// Contig of the window [pos, pos + span) of G when it is a placement on the
// reference, else PLACE_OFF_REFERENCE or PLACE_OUT_OF_RANGE.  span >= 1.
int32_t reference_place(const mica_reference &r, uint64_t pos, uint64_t span);

// SAM's reference-name rule: [0-9A-Za-z!#$%&+./:;?@^_|~-][0-9A-Za-z!#$%&*+./:;=?@^_|~-]*
bool sam_name_ok(const std::string &s);

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the value returned when
// the generator's state before the call is x.  Picks the stand-in base of an
// ambiguous byte (top two bits).
inline uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Base code of an A/C/G/T byte (either case), -1 for any other byte.
inline int base_code(uint8_t c)
{
    switch (c | 0x20) {
    case 'a': return 0;
    case 'c': return 1;
    case 'g': return 2;
    case 't': return 3;
    default: return -1;
    }
}

inline bool is_letter(uint8_t c) { return (c | 0x20) >= 'a' && (c | 0x20) <= 'z'; }

}  // namespace mica

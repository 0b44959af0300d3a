// Host-side batch of reads from FASTQ: the packed layout the search takes,
// plus what SAM records need (names, qualities, ambiguous offsets).  Shared
// by fastq.cpp (reading, the N filter) and sam.cpp (records).  No CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "mica.h"

struct mica_read_batch {
    std::vector<uint32_t> words;      // 2 bits per base, 16 bases per word, least significant first
    std::vector<uint64_t> word_off;   // n + 1
    std::vector<uint16_t> len;
    std::vector<uint8_t> k;
    std::string names;                // read i's name at names.c_str() + name_off[i], NUL-terminated
    std::vector<uint64_t> name_off;   // n + 1
    std::string quals;                // read i's qualities = quals[qual_off[i], qual_off[i] + len[i])
    std::vector<uint64_t> qual_off;   // n + 1
    std::vector<uint16_t> amb;        // read i's ambiguous offsets = amb[amb_off[i], amb_off[i + 1])
    std::vector<uint64_t> amb_off;    // n + 1
    uint64_t n_ambiguous_reads = 0;
    bool paired = false;

    uint64_t n() const { return len.size(); }
};

// Autotuner cache: best tile shape and modular product per shape bucket.
#pragma once
#include <string>
#include "internal.h"

namespace pe {

struct TuneEntry {
    uint32_t K = 0, wpb = 0;
    int variant = 0;
    uint32_t kslabs = 0, Tc = 0, tail = 0;   // item shape (0: the library's rule)
    double ms = 0.0;
};

std::string tune_key(const pe_poly *P, uint64_t T);
const TuneEntry *tune_lookup(const pe_poly *P, uint64_t T);   // nullptr when untuned
int run_variant(pe_poly *P, uint64_t T);                       // modular product for a plain run
int default_variant(uint64_t p);                               // fastest product for the prime's width

}  // namespace pe

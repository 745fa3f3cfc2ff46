// Autotuner cache: best tile shape and modular product per shape bucket.
#pragma once
#include <string>
#include "internal.h"

namespace pe {

struct TuneEntry {
    uint32_t K = 0, wpb = 0;
    int variant = 0;
    uint32_t kslabs = 0, Tc = 0, tail = 0;   // item shape (0: the library's rule)
    uint32_t method = 0;                       // 0: matrix method, 1: fast method (Sect. 2.3.1)
    double ms = 0.0;
};

std::string tune_key(const pe_poly *P, uint64_t T);
const TuneEntry *tune_lookup(const pe_poly *P, uint64_t T);   // nullptr when untuned
int run_variant(pe_poly *P, uint64_t T);                       // modular product for a plain run
int default_variant(uint64_t p);                               // fastest product for the prime's width
bool fast_applicable(uint64_t p, uint64_t T);                  // the fast method can run this (p, T)
// The matrix method without the tuner's choice of method (the public run
// dispatches to the fast method when the tuner measured it faster).
pe_status run_matrix(pe_poly *P, const uint64_t *beta, uint64_t T, uint64_t t0, uint64_t *out, void *stream);

}  // namespace pe

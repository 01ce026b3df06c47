// Internal definitions shared by the host compiler and the CUDA translation units.
#pragma once
#include <stdint.h>
#include <string>

#include "../../include/rv.h"

struct rv_quant {
  int kind;        // RV_Q_A or RV_Q_E
  int op;          // RV_LT .. RV_EQ
  uint64_t num;    // constant c = num / den (den = 1 for E)
  uint64_t den;
};

struct rv_formula {
  int n_quant;
  rv_quant q[2];
  int key_bits;
  int alphabet;
  int n_codes;
  int n_letters;
  int n_states;
  int q0;
  // comparison atoms "value ~ c" of the body: letter = code + n_base * (bit j: atom j holds)
  int n_base;                      // letters of the predicate byte alone (n_codes or 2^n_codes)
  int n_cmp;
  int cmp_op[RV_MAX_CMP];          // RV_LT .. RV_EQ
  uint32_t cmp_c[RV_MAX_CMP];
  uint64_t maps[RV_MAX_LETTERS];   // nibble s of maps[l] = delta(s, l)
  uint8_t labels[RV_MAX_STATES];   // lambda(s) as rv_verdict code
  std::string text;
};

// Thread-local error message handling (defined in formula.cpp).
rv_status rv_fail(rv_status st, const char* fmt, ...);

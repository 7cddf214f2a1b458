// Test-only exports of the library's host quantisers.
#include "quant.h"

extern "C" {
uint8_t quant_e4m3(float f) { return spider::to_e4m3(f); }
uint16_t quant_bf16(float f) { return spider::to_bf16(f); }
}

// Factorization entry points (filled in below the product driver).
#include "handle.h"

extern "C" {
int emul_dgetrf(emul_handle_t h, int, double*, int, int32_t*, int, int, int32_t*, emul_stats*) {
  return emul::set_error(h, EMUL_NOT_SUPPORTED, "not built yet");
}
int emul_dgetrs(emul_handle_t h, int, int, const double*, int, const int32_t*, double*, int) {
  return emul::set_error(h, EMUL_NOT_SUPPORTED, "not built yet");
}
int emul_dpotrf(emul_handle_t h, char, int, double*, int, int, int, int32_t*, emul_stats*) {
  return emul::set_error(h, EMUL_NOT_SUPPORTED, "not built yet");
}
int emul_dpotrs(emul_handle_t h, char, int, int, const double*, int, double*, int) {
  return emul::set_error(h, EMUL_NOT_SUPPORTED, "not built yet");
}
int emul_backward_error(emul_handle_t h, int, const double*, int, const double*, const double*, double*) {
  return emul::set_error(h, EMUL_NOT_SUPPORTED, "not built yet");
}
}

// rlb_internal.h -- helpers shared by the translation units of librlb (not part of the ABI).
#pragma once
#include <string>

namespace rlb {
// Checks the relaxation times of a problem statement (every tau > 0.5, tau_q <= 0
// meaning tau_v); returns RLB_OK or RLB_EINVAL with the reason in `why`.
int validate_taus(double tau_f, double tau_v, double tau_e, double tau_eps, double tau_q, int collision,
                  std::string& why);
// Records the message that rlb_last_error(NULL) returns (calls that take no handle).
void set_handleless_error(const std::string& msg);
}  // namespace rlb

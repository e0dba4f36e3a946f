// pflb_validate.cuh -- checks of a domain description and a mechanism shared
// by the entry points that take them (pflb_create_domain, pflb_set_mechanism,
// pflb_step_noalloc).  Defined in pflb_api.cu.
#pragma once

#include <string>

#include "../../include/pflb.h"

namespace pflb {

// Structural checks: lattice extent, precision, boundary kinds and their
// placement, positive physical scales and a finite, positive P0.
// PFLB_OK, or an error code with the reason in `msg`.
int validate_desc(const pflb_domain_desc& D, std::string& msg);

// Species count, reaction count, chemistry mode and positive species data.
int validate_mech(const pflb_mechanism& m, std::string& msg);

// Explicit-scheme limits at every temperature the description names (T_in,
// Ts_uniform, wall temperatures, T_max): BGK relaxation time above 1/2, the
// forward-Euler diffusion numbers of temperature, species and the solid at or
// below 1/(2 dim), the interface exchange number A_T a / eta^2 below 2 (and
// its solid side, A_T lambda (4/27) / (eta^2 (rho cp)_s), with a transported
// solid temperature), and an inlet speed below the lattice sound speed.  With m == nullptr (or
// K = 0) the gas is the single gas of the description (M0); otherwise the
// inlet mixture of m.  PFLB_ERR_UNSTABLE with the reason in `msg`.
int check_stability(const pflb_domain_desc& D, const pflb_mechanism* m, std::string& msg);

// Message for a status latched in the device status word.
const char* status_message(int status);

// The message pflb_last_error(NULL) returns on this host thread.
void set_global_error(const std::string& msg);

}  // namespace pflb

// Error reporting and parameter defaults.
#include <cstdio>
#include <string>

#include "common.cuh"

namespace pdfgb {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

pdf_status fail(pdf_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

pdf_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return PDF_ECUDA;
}

}  // namespace pdfgb

extern "C" const char* pdf_last_error(void) { return pdfgb::g_last_error.c_str(); }

extern "C" void pdf_model_params_default(pdf_model_params* p) {
  if (!p) return;
  p->dt = 1e-3;
  p->nu = 1e-3;
  p->Pi = 2e-3;
  p->c_phi = 2.0;
  p->closure = PDF_CLOSURE_GLM;
  p->tm_mode = PDF_TM_TURB;
  p->pressure = PDF_PRESSURE_CHANNEL;
  p->arith = PDF_ARITH_FX;
  // table "Constants for modeling the joint PDF of velocity and frequency"
  p->C1 = 1.85; p->C2 = 0.63; p->C3 = 5.0; p->C4 = 0.25; p->CT = 6.0; p->CL = 0.134;
  p->Ceta = 72.0; p->Cv = 1.4; p->gamma5 = 0.1; p->Comega1 = 0.5; p->Comega2 = 0.73;
  // eq. wall-GandC
  p->C0_slm = 3.5;
  // concentrated source: none; micromixing constants of the table of constants (ch. 5)
  p->src_x = 0.0; p->src_y = 0.0; p->src_r = 0.0;
  p->Cs = 0.02; p->Ct = 0.7;
  p->mix = PDF_MIX_IEM;
  p->reserved = 0;
}

// Host-only entry points of libchert: error text and the Thomsen conversion.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace chert {
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
}  // namespace chert

extern "C" const char* chert_last_error(void) { return chert::g_err; }

// Thomsen's (1986) parameters inverted for a VTI solid; quality factors per
// Voigt component as in the paper's Table 2 (Eq. 2: aI = aR / Q).
extern "C" int chert_thomsen_to_class(double vp0, double vs0, double eps, double delta,
                                      double gamma, double qp, double qs, double rho,
                                      double tilt, double azim, chert_class* out) {
    CHERT_REQUIRE(out != nullptr, "chert_thomsen_to_class: out is NULL");
    CHERT_REQUIRE(vp0 > 0 && vs0 > 0 && vp0 > vs0, "chert_thomsen_to_class: need vp0 > vs0 > 0");
    CHERT_REQUIRE(qp > 0 && qs > 0, "chert_thomsen_to_class: quality factors must be positive");
    const double a33 = vp0 * vp0, a44 = vs0 * vs0;
    const double a11 = a33 * (1.0 + 2.0 * eps);
    const double a66 = a44 * (1.0 + 2.0 * gamma);
    const double rad = (a33 - a44) * (a33 * (1.0 + 2.0 * delta) - a44);
    CHERT_REQUIRE(rad > 0.0, "chert_thomsen_to_class: delta=%g leaves no real a13", delta);
    const double a13 = sqrt(rad) - a44;
    const double aR[5] = {a11, a13, a33, a44, a66};
    const double q[5] = {qp, qp, qp, qs, qs};
    for (int i = 0; i < 5; i++) {
        out->aR[i] = aR[i];
        out->aI[i] = isinf(q[i]) ? 0.0 : aR[i] / q[i];
    }
    out->rho = rho;
    out->tilt = tilt;
    out->azim = azim;
    return CHERT_OK;
}

// Eq. 2 for media given as real moduli and a quality factor per component
// (the form of the paper's Table 2): aI = aR / Q, an infinite Q elastic.
extern "C" int chert_moduli_to_class(const double* aR, const double* q, double rho, double tilt, double azim,
                                     chert_class* out) {
    CHERT_REQUIRE(aR && q && out, "chert_moduli_to_class: NULL argument");
    for (int i = 0; i < 5; i++)
        CHERT_REQUIRE(q[i] > 0, "chert_moduli_to_class: Q of component %d is %g (must be positive)", i, q[i]);
    CHERT_REQUIRE(aR[2] > 0 && aR[3] > 0, "chert_moduli_to_class: a33 and a44 must be positive");
    for (int i = 0; i < 5; i++) {
        out->aR[i] = aR[i];
        out->aI[i] = isinf(q[i]) ? 0.0 : aR[i] / q[i];
    }
    out->rho = rho;
    out->tilt = tilt;
    out->azim = azim;
    return CHERT_OK;
}

// Batched form of chert_thomsen_to_class for per-cell media (host arrays).
extern "C" int chert_thomsen_to_classes(int64_t n, const double* vp0, const double* vs0, const double* eps,
                                        const double* delta, const double* gamma, const double* qp,
                                        const double* qs, const double* rho, const double* tilt,
                                        const double* azim, chert_class* out) {
    CHERT_REQUIRE(n >= 0 && vp0 && vs0 && eps && delta && gamma && qp && qs && rho && tilt && azim && out,
                  "chert_thomsen_to_classes: NULL argument");
    for (int64_t i = 0; i < n; ++i) {
        const int rc = chert_thomsen_to_class(vp0[i], vs0[i], eps[i], delta[i], gamma[i], qp[i], qs[i], rho[i],
                                              tilt[i], azim[i], out + i);
        if (rc) {
            char msg[512];
            snprintf(msg, sizeof(msg), "%s (class %lld)", chert_last_error(), (long long)i);
            chert::set_error("%s", msg);
            return rc;
        }
    }
    return CHERT_OK;
}

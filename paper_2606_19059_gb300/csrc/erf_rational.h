/* Generated by paper_2606_19059_gb300/fit_erf.py -- do not edit.
 *
 * FP64: erf(x)/x ~= P(z)/Q(z), z = 2x/ERF_RAT_X64 - 1, 0 <= x <= ERF_RAT_X64
 *       (Sec. 4: rational approximation of erf(x)/x, FMAs + one division).
 * FP32: erfcx(x) = e^{x^2} erfc(x) ~= t p(t), t = 1/(1 + ERFCX_C32 x),
 *       0 <= x <= ERFCX_X32.
 * Coefficients lowest degree first; *_MAXERR measured against 50-digit erf.
 */
#pragma once

#define ERF_RAT_X64 7.0
#define ERF_RAT_F64_N 14
#define ERF_RAT_F64_MAXERR 9.263e-14  /* absolute, on erf(x)/x, exact arithmetic */
#define ERF_RAT_F64_MAXERR_EVAL 6.212e-12  /* same, Horner in IEEE double */
static const double erf_rat_f64_p[14] = {
    2.85714073400538035854e-1,
    2.03660762557384976532,
    7.79395336783986220968,
    2.00371704103975344897e+1,
    3.78841871000466610409e+1,
    5.46795002577208587614e+1,
    6.12008135735338861635e+1,
    5.30730784025737531847e+1,
    3.51529124062755588824e+1,
    1.72398941288290492037e+1,
    5.90781657279309787753,
    1.26119093623723459311,
    1.26228241465486921011e-1,
    -9.75027678344811070817e-5,
};
static const double erf_rat_f64_q[14] = {
    1.0,
    8.12811308839581664428,
    3.44070669402358379901e+1,
    9.74084236267208698058e+1,
    2.02726448581838776942e+2,
    3.23968939011823316219e+2,
    4.05587564515708818204e+2,
    3.99951756583057138318e+2,
    3.08794517827907424656e+2,
    1.83376071411690659122e+2,
    8.10140471262104878466e+1,
    2.50922098735228202248e+1,
    4.85750785949956380934,
    4.4012071215943468606e-1,
};

#define ERFCX_X32 6.0
#define ERFCX_C32 0.5
#define ERFCX_F32_N 10
#define ERFCX_F32_MAXERR 3.970e-09  /* relative, on erfcx(x) */
static const double erfcx_f32_c[10] = {
    0.28200062013744914,
    0.2840617502035214,
    0.2288897727804148,
    0.2700693673383917,
    -0.22469336639707446,
    0.6528580672588761,
    -0.944474492531219,
    0.6321257783675847,
    -0.2086952530750035,
    0.027857751971397733,
};

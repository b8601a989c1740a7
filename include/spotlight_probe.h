/*
 * spotlight_probe.h -- measurement helper shipped with libspotlight.  The
 * paper has no counterpart: it exists to state the integer-add roofline of
 * the dedispersion kernel from a measurement on the running GPU.
 */
#ifndef SPOTLIGHT_PROBE_H
#define SPOTLIGHT_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Runs one CTA of 1024 threads per SM on the current device, each thread
 * executing `iters` x 24 independent 3-input 32-bit integer adds, and
 * reports the sustained rate in warp-lane add instructions per SM per clock
 * (the SM's own cycle counter, so the figure does not depend on the clock
 * frequency) and the SM count.  Allocates and frees a few KB of device
 * memory and synchronises the device.  Returns SP_OK, SP_EINVAL, SP_ENOMEM
 * or SP_ECUDA. */
int sp_probe_iadd3_rate(int iters, double *iadd3_per_sm_per_clk, int *num_sms);

#ifdef __cplusplus
}
#endif
#endif /* SPOTLIGHT_PROBE_H */

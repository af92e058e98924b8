"""FP64 CPU oracle for the Hadamard-spectral-code shading path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import or execute anything in this package.  The CUDA library never calls it,
and it never calls the CUDA library: the two share no code, headers, tables or
helpers.  The only thing both sides read is the seeded input module
``hsc_inputs`` (random draws and closed-form input spectra, none of the
method's arithmetic).

The oracle is plain and slow on purpose: float64 NumPy, no blocking, fusion or
reordering beyond what each definition states, so each function can be checked
against the paper by eye.  Modules:

* ``cmf``     colour matching functions, integration weights, sRGB, CIELAB,
              Delta E 76 / 94 / 2000 (Sec. 4.3 colour loss; Sec. 5.2 Lab)
* ``codec``   linear encoder/decoder and the blockwise Hadamard product
              (Eq. 4 and 6), the training objective (Eq. 8 and its four terms)
              and a projected-gradient fit of non-negative E, D
* ``shade``   spectral and latent deferred shading, k/3-pass form with
              reassembly, and a brute-force per-pixel loop form (Fig. 2b)
* ``metrics`` relative XYZ error and Delta E statistics
* ``quant``   storage rounding to bf16 / fp16 / fp8-e4m3 with per-channel
              scales

Parity status of each function is listed in its module header.  Functions
with no independent pin say "parity unpinned".
"""

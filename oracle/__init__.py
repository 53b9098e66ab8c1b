"""FP64 CPU oracle for the circulant inverse PFB (arXiv 2608.23441).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
anything in this package; only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` use it.  It shares no
code with the CUDA library: its only outside input is the seeded generator
module `paper_2608_23441_b300.synth` (random numbers, no method arithmetic).

Every function follows the paper's equations step by step, in float64, with
numpy's FFT (pocketfft) as the one library primitive.  No blocking, fusion or
reordering beyond what the cited definition states.

Modules
  pfb      window (Sec. 2.2, App. A), forward PFB (Eq. pfb / Eq. pfboperator),
           4-bit quantizer and byte packing (Sec. 4.3)
  ipfb     sub-filter eigenvalues (Sec. 3.1), circulant decorrelation
           (Eq. decorrelation), Wiener filter (Eq. wiener weights), analytic
           error spectra (App. B), dense brute-force references (App. C)
  upchan   up-channelization by long real FFTs (Sec. 4.3)
  ml       maximum-likelihood reconstruction with a time-domain prior
           (Eq. chi squared) by conjugate gradient
  net      learned CG preconditioner: conv net forward/backward, Adam,
           flexible CG (outside the paper; see its header)
  batched  many independent streams, one after another

Parity unpinned: the paper's end-to-end accuracy figures (Sec. 4.3) are
statistical results on a different quantizer step and mask scheme; they are
context only.  The learned preconditioner has no paper pin (its answers are checked
against plain CG on the same system).
"""

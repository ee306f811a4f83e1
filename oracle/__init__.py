"""FP64 CPU oracle for the autoencoder-compressed adjoint (arXiv 2304.04781).

TEST INFRASTRUCTURE, not part of the product: only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline / reference legs may import, call or execute anything
under oracle/.  The oracle shares no code with the CUDA path.

    wave.py     staggered leapfrog solver, discrete adjoint, Gauss-Newton HVP (Sec. 2, Sec. 4)
    codec.py    per-block autoencoder, normalisation, training step and LAMB (Sec. 3)
    codec_time.py  compression in time: 16-step strain windows of 2x8x8-node blocks,
                the optimal rank-k code inside a GELU network (Sec. 3.2, Sec. 1)
    revolve.py  binomial checkpointing step counts and schedule checker (Sec. 1)

Every function is pinned by tests/test_oracle_*.py against closed forms, invariants
and brute force, except the autoencoder-compressed gradient as a whole, whose parity
is unpinned beyond its pieces (no closed form exists for a trained codec's error).
"""

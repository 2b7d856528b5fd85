"""Plain, slow, FP64 CPU oracle for the urgency-served LiDAR pillar front end.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls, links or executes this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` may use it.  It shares no code with the CUDA library (no kernels, headers, helpers,
tables or constant generators); the only module both sides use is ``pp_synth`` (seeded inputs,
no method arithmetic).

Modules
-------
``oracle.pillars``  point -> pillar voxelisation, PointNet, BEV scatter, conv3x3 backbone
                    (the PointPillars front end that the paper's 3D-perception chains run,
                    Section 6 / Table 4).
``oracle.sched``    urgency (Eq. 2), stream-level binding with reservation (Section 4.4.3),
                    delayed launching (Section 4.4.4), batched/overlapped launch
                    synchronisation (Section 4.4.5), early chain exit (Section 4.3), the overall
                    deadline-miss ratio (Eq. 3), and a discrete-event simulation of the policy.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` (brute force on
hand-built inputs, closed forms, invariants, library routines for textbook sub-steps, and the
values printed in Table 2).  Parity unpinned: absolute GPU miss ratios and latencies (they
depend on timing).
"""

"""Plain, slow FP64 CPU oracle for the spaQR hot path (numpy/scipy).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  It shares no code with the GPU library (paper_2102_09878_gb300) and
never imports it; both are fed by the seeded generators in ``inputs/``.
"""

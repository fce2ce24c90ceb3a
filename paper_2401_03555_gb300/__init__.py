"""GB300-native interval-MDP abstraction builder (IMPaCT's construction step).

``paper_2401_03555_gb300.impact`` is the Python binding of the C-ABI library
``libimpact.so`` (hand-written sm_103a CUDA); ``workloads`` holds the seeded
problem generators. Importing the package loads nothing; the CUDA library is
loaded on first use of :mod:`.impact` and a missing library is an error.
"""

__all__ = ["impact", "workloads"]
